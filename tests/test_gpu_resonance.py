"""The resonance sweep (64 FFT bins, 2-33.5 Hz, around the compartment's 13 Hz response, sun-roof
pressure shaped by a synthetic PSD): GPU parity with the oracle on a small cabin, the linearity
the workload relies on (scaling the Dirichlet data scales the solution), and the full 64-bin
batch on the 282k-node cabin checked through true FP64 residuals."""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import fem, krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context, rel  # noqa: E402


def test_resonance_bins_match_oracle_on_small_cabin():
    prob = hi.cabin_problem(40, 22, 19)
    ctx = context(prob)
    fr = [2.0, 6.5, 13.0, 33.5]
    KM = fem.assemble_KM(prob.mesh)
    p, st = helm.helm_solve(ctx, fr, helm.make_opts("cocg", tol=1e-12, maxit=40000))
    for k, f in enumerate(fr):
        A, b = fem.system(prob, f, KM)
        x, ost = krylov.cocg(lambda v: A @ v, b, tol=1e-12, maxit=40000)
        assert st[k]["status"] == 0 and ost.converged
        assert rel(p[k].cpu().numpy(), x) <= 1e-9


def test_scaled_dirichlet_data_scales_the_solution():
    prob = hi.cabin_problem(40, 22, 19)
    f = 13.0
    a = complex(hi.resonance_spectrum(np.array([f]))[0])
    scaled = hi.Problem(prob.mesh, prob.beta, prob.dir_nodes, prob.p_dir * a)
    o = helm.make_opts("cocg", tol=1e-12, maxit=40000)
    p1, _ = helm.helm_solve(context(prob), [f], o)
    pa, _ = helm.helm_solve(context(scaled), [f], o)
    assert rel(pa[0].cpu().numpy(), a * p1[0].cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("mode", ["fp64", "dw"])
def test_full_resonance_batch(mode):
    prob = hi.cabin_problem(100, 56, 48)
    ctx = context(prob)
    fr = [float(f) for f in hi.resonance_freqs(64)]
    if mode == "fp64":
        o = helm.make_opts("cocg", tol=1e-10, maxit=40000, stall_window=15000)
    else:
        o = helm.make_opts("cocg", tol=1e-10, maxit=40000, mixed="dw", inner_tol=1e-12, inner_maxit=40000,
                           max_outer=20, stall_window=15000)
    p, st = helm.helm_solve(ctx, fr, o)
    assert all(s["status"] == 0 for s in st)
    for k in (0, 22, 63):  # 2, 13, 33.5 Hz
        A = helm.helm_assemble(ctx, fr[k])
        y = torch.empty_like(p[k])
        helm.helm_spmv(A, p[k].contiguous(), y)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(A.rhs - y) / torch.linalg.norm(A.rhs)).item() <= 1.01e-10
