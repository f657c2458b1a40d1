"""Failure detection without faulting the GPU: injected barrier timeout, injected
out-of-memory, non-finite data. After each failure the context must still solve normally."""
import os

import numpy as np
import pytest

import helm_inputs as hi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context  # noqa: E402


def solve_ok(ctx):
    p, st = helm.helm_solve(ctx, [100.0], helm.make_opts("cocg", tol=1e-10, maxit=20000))
    assert st[0]["status"] == 0 and st[0]["relres"] <= 1e-10


BARRIER_MODES = {
    "cocg_fp64": dict(solver="cocg"),
    "cocg_double_word_jacobi": dict(solver="cocg", mixed="dw", precond="jacobi", inner_tol=1e-12, inner_maxit=20000),
    "bicgstab": dict(solver="bicgstab"),
    "tfqmr_jacobi": dict(solver="tfqmr", precond="jacobi"),
}


@pytest.mark.parametrize("mode", list(BARRIER_MODES), ids=list(BARRIER_MODES))
def test_barrier_timeout_is_reported_and_the_context_survives(mode):
    # every persistent kernel (COCG in FP64 and double-word, BiCGSTAB, TFQMR's one-barrier state
    # machine) gives up at its bounded grid barrier and returns HELM_TIMEOUT
    ctx = context(hi.small_box_problem())
    os.environ["HELM_FAULT_INJECT"] = "barrier"
    try:
        p, st = helm.helm_solve(ctx, [100.0], helm.make_opts(tol=1e-10, maxit=20000, **BARRIER_MODES[mode]),
                                raise_on_fail=False)
    finally:
        del os.environ["HELM_FAULT_INJECT"]
    assert st[0]["status"] == helm.HELM_TIMEOUT
    assert b"timed out" in helm.LIB.helm_last_error()
    solve_ok(ctx)


def test_injected_out_of_memory_is_reported():
    ctx = context(hi.small_box_problem())
    os.environ["HELM_FAULT_INJECT"] = "oom"
    try:
        with pytest.raises(helm.HelmError) as ei:
            helm.helm_assemble(ctx, 100.0)
        p, st = helm.helm_solve(ctx, [100.0], helm.make_opts("cocg"), raise_on_fail=False)
    finally:
        del os.environ["HELM_FAULT_INJECT"]
    assert ei.value.status == helm.HELM_ERR_OOM
    solve_ok(ctx)


def test_non_finite_boundary_data_is_reported_as_nan():
    prob = hi.small_box_problem()
    bad = prob.p_dir.copy()
    bad[3] = np.nan
    ctx = context(hi.Problem(prob.mesh, prob.beta, prob.dir_nodes, bad))
    p, st = helm.helm_solve(ctx, [100.0], helm.make_opts("cocg", tol=1e-10, maxit=500), raise_on_fail=False)
    assert st[0]["status"] == helm.HELM_NAN
    ctx.set_boundary(torch.from_numpy(prob.beta).cuda(), torch.from_numpy(prob.dir_nodes).cuda(),
                     torch.from_numpy(prob.p_dir).cuda())
    solve_ok(ctx)


def test_argument_errors_before_device_work():
    ctx = context(hi.small_box_problem())
    o = helm.make_opts("gmres", restart=0)
    with pytest.raises(helm.HelmError) as ei:
        helm.helm_solve(ctx, [100.0], o)
    assert ei.value.status == helm.HELM_ERR_ARG
    bad_nodes = torch.tensor([0, ctx.n], dtype=torch.int32, device="cuda")
    with pytest.raises(helm.HelmError):
        ctx.set_boundary(None, bad_nodes, torch.zeros(2, dtype=torch.complex128, device="cuda"))
    solve_ok(ctx)
