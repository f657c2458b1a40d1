"""GPU checks of the double-word mixed mode (FP64 refinement around a COCG whose values are
pairs of floats, about 48 significand bits): the refined result meets the FP64 target, it is as
close to x* = A^-1 b as an FP64 COCG result, it needs about the FP64 step count, and it works
where the complex64 inner solve fails (171 Hz).

The oracle runs the same refinement in FP64 (oracle.krylov.cocg_ir), so the double-word path is
held to what any iterate at rel-res 1e-10 must satisfy (true FP64 residual, forward error next
to the FP64 solver's) and to the oracle's step count: within its rounding spread (the counts for
b and for three right-hand sides perturbed at 1e-14) widened by 5%.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import helm_inputs as hi
from oracle import fem, krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context, rel  # noqa: E402


def dw_opts(tol=1e-10, maxit=50000):
    return helm.make_opts("cocg", tol=tol, maxit=maxit, mixed="dw", inner_tol=1e-12, inner_maxit=maxit,
                          max_outer=20, stall_window=15000)


@pytest.mark.parametrize("prob_f", [
    (hi.small_box_problem(20, 16, 12), 100.0),
    (hi.cabin_problem(40, 22, 19), 150.0),
    (hi.cabin_problem(*hi.sweep_mesh_dims(171.0)), 171.0),
], ids=["box100", "cabin150", "sweep171"])
def test_dw_refinement(prob_f):
    prob, f = prob_f
    ctx = context(prob)
    p, st = helm.helm_solve(ctx, [f], dw_opts())
    A, b = fem.system(prob, f)
    g = p[0].cpu().numpy()
    assert st[0]["status"] == 0, st
    assert st[0]["outer"] >= 1, st                       # no fallback to FP64 COCG
    assert st[0]["iterations_c64"] == st[0]["iterations"]
    assert np.linalg.norm(b - A @ g) / np.linalg.norm(b) <= 1e-10
    counts = []
    for sd in (0, 1, 2, 3):
        rhs = b
        if sd:
            rng = np.random.default_rng(sd)
            rhs = b + (rng.standard_normal(len(b)) + 1j * rng.standard_normal(len(b))) * 1e-14 * np.abs(b).max()
        _, ost, outer = krylov.cocg_ir(lambda v: A @ v, rhs, tol=1e-10, inner_maxit=50000, maxit=50000,
                                       stall=15000)
        assert ost.converged and outer == 1
        counts.append(ost.iterations)
    assert 0.95 * min(counts) - 1 <= st[0]["iterations"] <= 1.05 * max(counts) + 1, (st[0], counts)
    xs = spl.spsolve(A.tocsc(), b)
    p64, _ = helm.helm_solve(ctx, [f], helm.make_opts("cocg", tol=1e-10, maxit=50000))
    e_dw, e_64 = rel(g, xs), rel(p64[0].cpu().numpy(), xs)
    assert e_dw <= max(10 * e_64, 1e-9), (e_dw, e_64)


def test_dw_tight_tolerance_against_exact_solution():
    # at rel-res 1e-13 the double-word inner solve alone cannot finish; refinement must
    prob = hi.small_box_problem(20, 16, 12)
    ctx = context(prob)
    p, st = helm.helm_solve(ctx, [100.0], dw_opts(tol=1e-13))
    A, b = fem.system(prob, 100.0)
    xs = spl.spsolve(A.tocsc(), b)
    assert st[0]["status"] == 0 and st[0]["outer"] >= 1
    assert rel(p[0].cpu().numpy(), xs) <= 1e-9


def test_dw_batch_of_different_meshes():
    freqs = [20.0, 180.0, 240.0, 300.0]
    probs = [hi.cabin_problem(*hi.sweep_mesh_dims(f)) for f in freqs]
    ctxs = [context(pr) for pr in probs]
    ps, st = helm.helm_solve_batch(ctxs, freqs, dw_opts())
    for k, (pr, f) in enumerate(zip(probs, freqs)):
        A, b = fem.system(pr, f)
        g = ps[k].cpu().numpy()
        assert st[k]["status"] == 0 and st[k]["outer"] >= 1, st[k]
        assert np.linalg.norm(b - A @ g) / np.linalg.norm(b) <= 1e-10


def test_dw_zero_rhs_and_nonconvergence():
    mesh = hi.Mesh(1, 1, 1, 0.3, 0.2, 0.1)
    zero = hi.Problem(mesh, np.full(6, 0.02 + 0.01j), np.array([7], dtype=np.int32), np.array([0.0 + 0.0j]))
    p, st = helm.helm_solve(context(zero), [500.0], dw_opts())
    assert st[0]["status"] == 0 and st[0]["iterations"] == 0
    assert np.all(p[0].cpu().numpy() == 0)
    ctx = context(hi.small_box_problem())
    p, st = helm.helm_solve(ctx, [100.0], dw_opts(maxit=9), raise_on_fail=False)
    assert st[0]["status"] == helm.HELM_NOT_CONVERGED and st[0]["iterations"] <= 9
    assert np.isfinite(p[0].cpu().numpy()).all()
