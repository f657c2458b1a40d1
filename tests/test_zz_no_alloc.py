"""GPU test of helm_reduce_noalloc, the reduction that allocates no device memory.

It serves callers that cannot call cudaMalloc while they run (a fixed, pre-reserved memory
budget, or loops that cannot take cudaMalloc's implicit device synchronisation). Its result must
agree with helm_reduce within the reduction tolerance of the other tests, on two calls in a row
(the static scratch array keeps the previous call's contents), both in a fresh process and after
the other tests. The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import helm_inputs as hi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402


def c_abi(name, op, x, y):
    out = (ctypes.c_double * 2)()
    st = getattr(helm.LIB, name)(op, x.numel(), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()) if y is not None else None, out,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == helm.HELM_OK, helm.LIB.helm_last_error()
    return complex(out[0], out[1])


@pytest.mark.parametrize("n", [1, 4097, 1_000_003])
def test_noalloc_reduction_matches_allocating_one_twice(n):
    x = torch.from_numpy(hi.random_complex(n, seed=11)).cuda()
    y = torch.from_numpy(hi.random_complex(n, seed=12)).cuda()
    mag = float((x.abs() * y.abs()).sum())
    for op, yy in ((0, y), (1, y), (2, None)):
        ref = c_abi("helm_reduce", op, x, yy)
        first = c_abi("helm_reduce_noalloc", op, x, yy)
        second = c_abi("helm_reduce_noalloc", op, x, yy)
        scale = mag if op != 2 else abs(ref)
        assert abs(first - ref) <= 1e-14 * scale
        assert abs(second - ref) <= 1e-14 * scale
        assert first == second


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = 16_777_216 + 1
    out = (ctypes.c_double * 2)()
    x = torch.zeros(1, dtype=torch.complex128, device="cuda")
    st = helm.LIB.helm_reduce_noalloc(2, n, ctypes.c_void_p(x.data_ptr()), None, out, None)
    assert st == helm.HELM_ERR_ARG
    assert b"16777216" in helm.LIB.helm_last_error()


def test_noalloc_needs_no_device_allocation():
    # with every device allocation of the library failing (host-side injection, no GPU fault),
    # helm_reduce reports HELM_ERR_OOM while helm_reduce_noalloc still gives the same result
    import os
    n = 50_001
    x = torch.from_numpy(hi.random_complex(n, seed=21)).cuda()
    y = torch.from_numpy(hi.random_complex(n, seed=22)).cuda()
    ref = c_abi("helm_reduce", 1, x, y)
    before = c_abi("helm_reduce_noalloc", 1, x, y)
    os.environ["HELM_FAULT_INJECT"] = "oom"
    try:
        out = (ctypes.c_double * 2)()
        st = helm.LIB.helm_reduce(1, n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), out,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == helm.HELM_ERR_OOM
        during = c_abi("helm_reduce_noalloc", 1, x, y)
    finally:
        del os.environ["HELM_FAULT_INJECT"]
    assert during == before
    assert abs(during - ref) <= 1e-14 * float((x.abs() * y.abs()).sum())
