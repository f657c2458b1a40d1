"""GPU checks of the adjoint gradient at the adjoint workload's sizes (282,093-node cabin, 64
frequencies 20-300 Hz, listener sphere r = 0.15 m at (1.6, 0.4, 0.9), 2,688 seat admittances):

  * the hand-written adjoint against central differences of the listener objective through the
    GPU forward solve (h = 1e-6, forward solves at rel-res 1e-13) on 20 seeded seat faces and
    5 seeded sun-roof nodes;
  * on the 20x16x12 box of the single-frequency workload, against the oracle's adjoint with the
    solves done by dense LU (the plain definition), to rel-L2 <= 1e-9;
  * the 64-frequency gradient through the benchmark's main mode (double-word inner COCG, FP64
    refinement, symmetric Jacobi) against the FP64 COCG gradient of the same sweep.
"""
import numpy as np
import pytest

import bench
import helm_inputs as hi
from oracle import adjoint

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context, rel  # noqa: E402


def test_adjoint_central_differences_at_cabin_size():
    prob = hi.cabin_problem(100, 56, 48)
    ctx = context(prob)
    freqs = [60.0, 150.0]
    w = torch.from_numpy(hi.listener_weights(prob.mesh)).cuda()
    o = helm.make_opts("cocg", tol=1e-13, maxit=60000, stall_window=bench.STALL)
    p, st = helm.helm_solve(ctx, freqs, o)
    J, gb, gd = helm.helm_adjoint_grad(ctx, freqs, o, p, w)
    gb, gd = gb.cpu().numpy(), gd.cpu().numpy()
    nodes = torch.from_numpy(prob.dir_nodes).cuda()

    def objective(beta, pdir):
        ctx.set_boundary(torch.from_numpy(beta).cuda(), nodes, torch.from_numpy(pdir).cuda())
        pp, s2 = helm.helm_solve(ctx, freqs, o)
        return float((w[None, :] * pp.abs() ** 2).sum().item())

    assert abs(objective(prob.beta, prob.p_dir) - J) <= 1e-10 * J
    rng = np.random.default_rng(0)
    h = 1e-6
    seats = np.flatnonzero(prob.beta != 0)
    assert len(seats) == 2688
    for e in rng.choice(seats, 20, replace=False):
        for unit in (1.0, 1j):
            bp, bm = prob.beta.copy(), prob.beta.copy()
            bp[e] += h * unit
            bm[e] -= h * unit
            fd = (objective(bp, prob.p_dir) - objective(bm, prob.p_dir)) / (2 * h)
            an = gb[e].real if unit == 1.0 else gb[e].imag
            # central differences carry an absolute error set by the solve accuracy over h, so the
            # bound is relative to the gradient's scale
            assert abs(fd - an) <= 1e-5 * np.abs(gb).max(), (e, unit, fd, an)
    for t in rng.choice(len(prob.dir_nodes), 5, replace=False):
        for unit in (1.0, 1j):
            pp_, pm_ = prob.p_dir.copy(), prob.p_dir.copy()
            pp_[t] += h * unit
            pm_[t] -= h * unit
            fd = (objective(prob.beta, pp_) - objective(prob.beta, pm_)) / (2 * h)
            an = gd[t].real if unit == 1.0 else gd[t].imag
            assert abs(fd - an) <= 1e-5 * np.abs(gd).max(), (t, unit, fd, an)


def test_adjoint_matches_dense_oracle_on_the_box():
    prob = hi.small_box_problem(20, 16, 12)
    ctx = context(prob)
    freqs = [100.0, 150.0]
    w = hi.listener_weights(prob.mesh, centre=(0.5, 0.4, 0.3), radius=0.15)
    assert (w > 0).sum() > 1
    o = helm.make_opts("cocg", tol=1e-13, maxit=20000, stall_window=bench.STALL)
    p, st = helm.helm_solve(ctx, freqs, o)
    assert all(s["status"] == 0 for s in st)
    J, gb, gd = helm.helm_adjoint_grad(ctx, freqs, o, p, torch.from_numpy(w).cuda())
    Jr, gbr, gdr, _ = adjoint.objective_and_gradient(prob, freqs, w, dense=True)
    assert abs(J - Jr) <= 1e-10 * Jr
    assert rel(gb.cpu().numpy(), gbr) <= 1e-9
    assert rel(gd.cpu().numpy(), gdr) <= 1e-9


def test_adjoint_sweep_main_mode_matches_fp64():
    prob = hi.cabin_problem(100, 56, 48)
    ctx = context(prob)
    freqs = list(np.geomspace(20.0, 300.0, 64))
    w = torch.from_numpy(hi.listener_weights(prob.mesh)).cuda()
    out = {}
    for name, o in (("fp64", helm.make_opts("cocg", tol=1e-12, maxit=60000, stall_window=bench.STALL)),
                    ("main", helm.make_opts("cocg", tol=1e-12, maxit=60000, mixed="dw", inner_tol=1e-12,
                                            inner_maxit=60000, max_outer=20, stall_window=bench.STALL,
                                            precond="jacobi"))):
        p, st = helm.helm_solve(ctx, freqs, o)
        assert all(s["status"] == 0 for s in st), name
        out[name] = helm.helm_adjoint_grad(ctx, freqs, o, p, w)
    (J1, gb1, gd1), (J2, gb2, gd2) = out["fp64"], out["main"]
    assert abs(J2 - J1) <= 1e-9 * J1
    assert (torch.linalg.norm(gb2 - gb1) / torch.linalg.norm(gb1)).item() <= 1e-7
    assert (torch.linalg.norm(gd2 - gd1) / torch.linalg.norm(gd1)).item() <= 1e-7
