"""Shared-mesh multi-frequency product (helm_spmv_multi) against the CPU oracle: Y[f] = A(f) X[f]
with A(f) the oracle's eliminated system matrix, for batches that span one and two passes of 8
frequencies, in complex128 and complex64; and against the single-frequency product at full size."""
import numpy as np
import pytest

import helm_inputs as hi
from oracle import fem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context  # noqa: E402

FREQS = [0.0, 50.0, 150.0, 230.0, 333.3, 500.0, 17.0, 90.0, 400.0]  # 9: a full pass of 8 and one more

CASES = [
    ("box100", hi.small_box_problem()),
    ("ragged_cabin", hi.cabin_problem(13, 7, 5)),
    ("single_brick", hi.Problem(hi.Mesh(1, 1, 1, 0.3, 0.2, 0.1), np.full(6, 0.02 + 0.01j),
                                np.array([7], dtype=np.int32), np.array([1.0 + 0.5j]))),
]


@pytest.mark.parametrize("name,prob", CASES, ids=[c[0] for c in CASES])
def test_multi_frequency_product_matches_oracle(name, prob):
    ctx = context(prob)
    n = ctx.n
    X = np.stack([hi.random_complex(n, seed=11 + f) for f in range(len(FREQS))])
    KM = fem.assemble_KM(prob.mesh)
    refs, bounds = [], []
    for f, fr in enumerate(FREQS):
        A, _ = fem.system(prob, fr, KM)
        refs.append(A @ X[f])
        bounds.append(abs(A) @ np.abs(X[f]))
    for prec, tol in ((helm.HELM_C128, 1e-13), (helm.HELM_C64, 64 * 2.0 ** -24)):
        S = helm.helm_assemble_shared(ctx, prec)
        dt = torch.complex128 if prec == helm.HELM_C128 else torch.complex64
        Xg = torch.from_numpy(X).to(dt).cuda().contiguous()
        Yg = torch.empty_like(Xg)
        helm.helm_spmv_multi(S, FREQS, Xg, Yg)
        torch.cuda.synchronize()
        Y = Yg.cpu().numpy().astype(np.complex128)
        for f in range(len(FREQS)):
            err = np.abs(Y[f] - refs[f])
            assert np.all(err <= tol * bounds[f] + 1e-30), (prec, FREQS[f], float((err / (bounds[f] + 1e-300)).max()))
        S.close()


def test_multi_frequency_product_equals_assembled_product_at_full_size():
    """2,203,161-node cabin with its boundary data: every frequency of a 12-frequency batch equals
    helm_spmv on the matrix helm_assemble builds for that frequency (the same entries, combined
    per frequency), to rounding."""
    prob = hi.cabin_problem(200, 112, 96)
    ctx = context(prob)
    freqs = list(np.geomspace(100.0, 400.0, 12))
    S = helm.helm_assemble_shared(ctx, helm.HELM_C128)
    g = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn(len(freqs), ctx.n, dtype=torch.complex128, device="cuda", generator=g)
    Y = torch.empty_like(X)
    helm.helm_spmv_multi(S, freqs, X, Y)
    y1 = torch.empty(ctx.n, dtype=torch.complex128, device="cuda")
    for f, fr in enumerate(freqs):
        A = helm.helm_assemble(ctx, fr, with_rhs=False, fmt=helm.HELM_FMT_DIA27)
        helm.helm_spmv(A, X[f].contiguous(), y1)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(Y[f] - y1) / torch.linalg.norm(y1)).item() <= 1e-14, fr
        del A
    S.close()


def test_multi_frequency_argument_errors():
    ctx = context(hi.small_box_problem(6, 4, 3))
    S = helm.helm_assemble_shared(ctx, helm.HELM_C128)
    X = torch.zeros(2, ctx.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(helm.HelmError):  # X and Y overlap
        helm._check(helm.LIB.helm_spmv_multi(S.handle, (helm.ctypes.c_double * 2)(1.0, 2.0), 2,
                                             helm._ptr(X), helm._ptr(X), None))
    # partial overlap: Y starts inside X (one frequency), valid frequencies
    X3 = torch.zeros(3, ctx.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(helm.HelmError):
        helm._check(helm.LIB.helm_spmv_multi(S.handle, (helm.ctypes.c_double * 2)(1.0, 2.0), 2,
                                             helm._ptr(X3), helm._ptr(X3[1:]), None))
    # adjacent, not overlapping: accepted
    helm._check(helm.LIB.helm_spmv_multi(S.handle, (helm.ctypes.c_double * 1)(1.0), 1,
                                         helm._ptr(X3[0:1]), helm._ptr(X3[1:2]), None))
    torch.cuda.synchronize()
    with pytest.raises(helm.HelmError):  # negative frequency
        helm._check(helm.LIB.helm_spmv_multi(S.handle, (helm.ctypes.c_double * 1)(-5.0), 1,
                                             helm._ptr(X3[0:1]), helm._ptr(X3[2:3]), None))
    # an empty batch is a no-op
    helm._check(helm.LIB.helm_spmv_multi(S.handle, (helm.ctypes.c_double * 1)(1.0), 0, None, None, None))
    S.close()


@pytest.mark.parametrize("name,prob", CASES, ids=[c[0] for c in CASES])
def test_interleaved_product_matches_oracle(name, prob):
    # node-major X, Y ([n][F]): the same products as the frequency-major form, against the oracle
    ctx = context(prob)
    n = ctx.n
    for prec, tol, nfs in ((helm.HELM_C128, 1e-13, (1, 2, 4, 8)), (helm.HELM_C64, 64 * 2.0 ** -24, (2, 4, 8))):
        S = helm.helm_assemble_shared(ctx, prec)
        dt = torch.complex128 if prec == helm.HELM_C128 else torch.complex64
        for F in nfs:
            freqs = FREQS[:F]
            X = np.stack([hi.random_complex(n, seed=31 + f) for f in range(F)], axis=1)  # [n][F]
            Xg = torch.from_numpy(X).to(dt).cuda().contiguous()
            Yg = torch.empty_like(Xg)
            helm.helm_spmv_multi_interleaved(S, freqs, Xg, Yg)
            torch.cuda.synchronize()
            Y = Yg.cpu().numpy().astype(np.complex128)
            KM = fem.assemble_KM(prob.mesh)
            for f, fr in enumerate(freqs):
                A, _ = fem.system(prob, fr, KM)
                ref = A @ X[:, f]
                bound = abs(A) @ np.abs(X[:, f])
                err = np.abs(Y[:, f] - ref)
                assert np.all(err <= tol * bound + 1e-30), (prec, F, fr)
        S.close()


def test_interleaved_product_arguments():
    ctx = context(hi.small_box_problem(6, 4, 3))
    S = helm.helm_assemble_shared(ctx, helm.HELM_C64)
    X = torch.zeros(ctx.n, 3, dtype=torch.complex64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(helm.HelmError):  # 3 frequencies: not a supported block width
        helm._check(helm.LIB.helm_spmv_multi_interleaved(S.handle, (helm.ctypes.c_double * 3)(1.0, 2.0, 3.0), 3,
                                                          helm._ptr(X), helm._ptr(Y), None))
    X4 = torch.zeros(ctx.n * 4 + 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(helm.HelmError):  # misaligned (8-byte offset)
        helm._check(helm.LIB.helm_spmv_multi_interleaved(S.handle, (helm.ctypes.c_double * 4)(1.0, 2.0, 3.0, 4.0), 4,
                                                          helm._ptr(X4[1:]), helm._ptr(Y), None))
    S.close()

