"""Parity at the benchmark's full size and launch configuration, and a full-size adjoint check.

The 256-frequency sweep is solved exactly as bench.py times its main leg (one helm_solve_batch
call, same options: double-word inner COCG, FP64 refinement, symmetric Jacobi). Systems small enough for the oracle are compared with it one by one; every sampled large
system is checked through its true FP64 residual computed by a different kernel (helm_spmv on the
CSR matrix)."""
import numpy as np
import pytest

import bench
import helm_inputs as hi
from oracle import fem, krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context, rel  # noqa: E402


def true_relres(ctx, f, x):
    A = helm.helm_assemble(ctx, f)
    y = torch.empty_like(x)
    helm.helm_spmv(A, x.contiguous(), y)
    torch.cuda.synchronize()
    return (torch.linalg.norm(A.rhs - y) / torch.linalg.norm(A.rhs)).item()


def test_full_sweep_in_the_benchmark_configuration():
    freqs = hi.sweep_freqs(256)
    probs = [hi.cabin_problem(*hi.sweep_mesh_dims(f)) for f in freqs]
    ctxs = [context(p) for p in probs]
    # the benchmark's main leg: double-word inner COCG with FP64 refinement, symmetric Jacobi
    opts = bench.dw_opts(helm, precond="jacobi")
    ps, st = helm.helm_solve_batch(ctxs, freqs, opts)
    assert all(s["status"] == 0 for s in st)
    assert all(s["outer"] >= 1 for s in st)  # no system fell back to FP64 COCG
    # oracle (FP64 symmetric-Jacobi COCG), one by one, on systems it solves in seconds
    for k in (0, 60, 120, 150):
        A, b = fem.system(probs[k], freqs[k])
        Ah, sc, w = krylov.sym_jacobi(A)
        y, ost = krylov.cocg(lambda v: Ah @ v, sc * b, tol=1e-10, maxit=45000, stall=bench.STALL, weights=w)
        x = sc * y
        g = ps[k].cpu().numpy()
        assert np.linalg.norm(b - A @ g) / np.linalg.norm(b) <= 1e-10
        # inner double-word steps against FP64 steps: within 25% (median +4% on the sweep)
        assert 0.75 * ost.iterations - 2 <= st[k]["iterations"] <= 1.25 * ost.iterations + 2, (k, st[k], ost.iterations)
        assert rel(g, x) <= 1e-6
    # large systems: true residual through an independent kernel
    for k in (200, 230, 240, 245, 250, 255):
        assert true_relres(ctxs[k], freqs[k], ps[k]) <= 1.01e-10, k


def test_adjoint_central_differences_at_cabin_size():
    """282,093-node cabin: the hand-written adjoint gradient against central differences of the
    listener objective through the GPU forward solve (h = 1e-6, forward solves at rel-res 1e-13)."""
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
    faces = rng.choice(np.flatnonzero(prob.beta != 0), 6, replace=False)
    for e in faces:
        for unit in (1.0, 1j):
            bp, bm = prob.beta.copy(), prob.beta.copy()
            bp[e] += h * unit
            bm[e] -= h * unit
            fd = (objective(bp, prob.p_dir) - objective(bm, prob.p_dir)) / (2 * h)
            an = gb[e].real if unit == 1.0 else gb[e].imag
            # central differences carry an absolute error set by the solve accuracy over h, so the
            # bound is relative to the gradient's scale
            assert abs(fd - an) <= 1e-5 * np.abs(gb).max(), (e, unit, fd, an)
    for t in rng.choice(len(prob.dir_nodes), 3, replace=False):
        for unit in (1.0, 1j):
            pp_, pm_ = prob.p_dir.copy(), prob.p_dir.copy()
            pp_[t] += h * unit
            pm_[t] -= h * unit
            fd = (objective(prob.beta, pp_) - objective(prob.beta, pm_)) / (2 * h)
            an = gd[t].real if unit == 1.0 else gd[t].imag
            assert abs(fd - an) <= 1e-5 * np.abs(gd).max(), (t, unit, fd, an)
