"""GPU parity of assembly, SpMV and reductions against the CPU oracle (through the C ABI)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import helm_inputs as hi
from oracle import fem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2112_00087_gb300 import helm  # noqa: E402
from tests.gpu_util import context, dia_to_scipy, gpu_matrix, rel  # noqa: E402


CASES = [
    ("box100", hi.small_box_problem(), 100.0),
    ("ragged_cabin", hi.cabin_problem(13, 7, 5), 230.0),
    ("cabin_mid", hi.cabin_problem(40, 22, 19), 150.0),
    ("single_brick", hi.Problem(hi.Mesh(1, 1, 1, 0.3, 0.2, 0.1), np.full(6, 0.02 + 0.01j),
                                np.array([7], dtype=np.int32), np.array([1.0 + 0.5j])), 500.0),
]


@pytest.mark.parametrize("name,prob,f", CASES, ids=[c[0] for c in CASES])
def test_assembly_matches_oracle(name, prob, f):
    ctx = context(prob)
    A, S, b = gpu_matrix(ctx, f)
    K, M = fem.assemble_KM(prob.mesh)
    Ared, bref = fem.system(prob, f, (K, M))
    # pattern: bit-exact against the oracle's assembled 27-point pattern
    Kc = K.tocsr()
    Kc.sort_indices()
    assert np.array_equal(S.indptr, Kc.indptr) and np.array_equal(S.indices, Kc.indices)
    # values: the closed-form product and the quadrature scatter-add differ only by rounding
    D = (S - Ared).tocoo()
    scale = abs(Ared).max()
    assert (abs(D.data).max() if D.nnz else 0.0) <= 1e-14 * scale
    assert np.max(np.abs(b - bref)) <= 1e-14 * max(np.max(np.abs(bref)), 1e-300) + 1e-300
    # the GPU matrix is bitwise symmetric
    assert abs(S - S.T).max() == 0.0


@pytest.mark.parametrize("name,prob,f", CASES, ids=[c[0] for c in CASES])
def test_spmv_c128_and_c64(name, prob, f):
    ctx = context(prob)
    A, S, _ = gpu_matrix(ctx, f)
    x = hi.random_complex(ctx.n, seed=5)
    xg = torch.from_numpy(x).cuda()
    y = torch.empty_like(xg)
    helm.helm_spmv(A, xg, y)
    torch.cuda.synchronize()
    Aref, _ = fem.system(prob, f)
    yref = Aref @ x
    absbound = abs(Aref) @ np.abs(x)
    err = np.abs(y.cpu().numpy() - yref)
    assert np.all(err <= 1e-13 * absbound + 1e-300)
    assert rel(y.cpu().numpy(), yref) <= 1e-13
    # complex64 matrix: FP32 values and accumulation, bounded by rounding of each product
    A32 = helm.helm_assemble(ctx, f, helm.HELM_C64, with_rhs=False)
    x32 = xg.to(torch.complex64)
    y32 = torch.empty_like(x32)
    helm.helm_spmv(A32, x32, y32)
    torch.cuda.synchronize()
    u = 2.0 ** -24
    err32 = np.abs(y32.cpu().numpy().astype(np.complex128) - yref)
    assert np.all(err32 <= 64 * u * absbound + 1e-30)


@pytest.mark.parametrize("name,prob,f", CASES, ids=[c[0] for c in CASES])
def test_dia27_layout_assembly_and_spmv(name, prob, f):
    """Slot-major 27-point layout: same matrix as the oracle, padded slots zero, SpMV parity."""
    ctx = context(prob)
    A = helm.helm_assemble(ctx, f, fmt=helm.HELM_FMT_DIA27)
    v27 = A.dia27()
    m = prob.mesh
    # slots whose neighbour lies outside the lattice hold zero
    vv = v27.cpu().numpy()
    n = ctx.n
    r = np.arange(n)
    i, j, l = r % (m.nx + 1), (r // (m.nx + 1)) % (m.ny + 1), r // ((m.nx + 1) * (m.ny + 1))
    for k in range(27):
        di, dj, dl = k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1
        outside = (i + di < 0) | (i + di > m.nx) | (j + dj < 0) | (j + dj > m.ny) | (l + dl < 0) | (l + dl > m.nz)
        assert np.all(vv[k][outside] == 0)
    S = dia_to_scipy(v27, m)
    Aref, bref = fem.system(prob, f)
    assert abs(S - Aref).max() <= 1e-14 * abs(Aref).max()
    assert np.max(np.abs(A.rhs.cpu().numpy() - bref)) <= 1e-14 * np.max(np.abs(bref))
    x = hi.random_complex(n, seed=9)
    xg = torch.from_numpy(x).cuda()
    y = torch.empty_like(xg)
    helm.helm_spmv(A, xg, y)
    torch.cuda.synchronize()
    yref = Aref @ x
    absbound = abs(Aref) @ np.abs(x)
    assert np.all(np.abs(y.cpu().numpy() - yref) <= 1e-13 * absbound + 1e-300)
    A32 = helm.helm_assemble(ctx, f, helm.HELM_C64, with_rhs=False, fmt=helm.HELM_FMT_DIA27)
    x32 = xg.to(torch.complex64)
    y32 = torch.empty_like(x32)
    helm.helm_spmv(A32, x32, y32)
    torch.cuda.synchronize()
    err32 = np.abs(y32.cpu().numpy().astype(np.complex128) - yref)
    assert np.all(err32 <= 64 * 2.0 ** -24 * absbound + 1e-30)


@pytest.mark.parametrize("n", [1, 255, 1000, 1 << 20, (1 << 20) + 77])
def test_reductions_match_exact_sums(n):
    x = hi.random_complex(n, seed=1)
    y = hi.random_complex(n, seed=2)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    dotc = helm.helm_reduce(0, xg, yg)
    dotu = helm.helm_reduce(1, xg, yg)
    nrm = helm.helm_reduce(2, xg).real
    pc, pu = np.conj(x) * y, x * y
    ref_c = complex(math.fsum(pc.real), math.fsum(pc.imag))
    ref_u = complex(math.fsum(pu.real), math.fsum(pu.imag))
    ref_n = math.sqrt(math.fsum(np.abs(x) ** 2))
    mag = np.sum(np.abs(x) * np.abs(y))
    assert abs(dotc - ref_c) <= 1e-14 * mag
    assert abs(dotu - ref_u) <= 1e-14 * mag
    assert abs(nrm - ref_n) <= 1e-14 * ref_n
    # fixed-order reduction: repeated calls are bitwise identical
    assert helm.helm_reduce(0, xg, yg) == dotc


def test_full_size_operator_properties():
    """2,203,161-node lattice (the mixed-precision workload): properties that hold at any size.

    Rigid box, no Dirichlet data: A(f) = K - k^2 M. For a tensor-cosine v, K v = lam_h M v
    exactly, so A(f1) v = (lam_h - k1^2) / (k2^2 - k1^2) (A(f1) v - A(f2) v); and A is symmetric:
    x^T (A y) = y^T (A x).
    """
    mesh = hi.Mesh(200, 112, 96, *hi.CABIN)
    ctx = helm.Context(mesh.nx, mesh.ny, mesh.nz, mesh.Lx, mesh.Ly, mesh.Lz)
    assert ctx.n == 2203161 and ctx.nnz == mesh.nnz27
    f1, f2 = 150.0, 260.0
    A1 = helm.helm_assemble(ctx, f1, with_rhs=False)
    A2 = helm.helm_assemble(ctx, f2, with_rhs=False)
    dev = "cuda"
    i = torch.arange(mesh.nx + 1, device=dev, dtype=torch.float64)
    j = torch.arange(mesh.ny + 1, device=dev, dtype=torch.float64)
    l = torch.arange(mesh.nz + 1, device=dev, dtype=torch.float64)
    a, b_, c = 3, 2, 5
    v = (torch.cos(math.pi * c * l / mesh.nz)[:, None, None] * torch.cos(math.pi * b_ * j / mesh.ny)[None, :, None]
         * torch.cos(math.pi * a * i / mesh.nx)[None, None, :]).reshape(-1).to(torch.complex128).contiguous()

    def lam(q, n, h):
        th = math.pi * q / n
        return (6.0 / h ** 2) * (1 - math.cos(th)) / (2 + math.cos(th))
    lh = lam(a, mesh.nx, mesh.Lx / mesh.nx) + lam(b_, mesh.ny, mesh.Ly / mesh.ny) + lam(c, mesh.nz, mesh.Lz / mesh.nz)
    k1, k2 = 2 * math.pi * f1 / hi.C_SOUND, 2 * math.pi * f2 / hi.C_SOUND
    y1, y2 = torch.empty_like(v), torch.empty_like(v)
    helm.helm_spmv(A1, v, y1)
    helm.helm_spmv(A2, v, y2)
    pred = (lh - k1 * k1) / (k2 * k2 - k1 * k1) * (y1 - y2)
    assert (torch.linalg.norm(y1 - pred) / torch.linalg.norm(y1)).item() <= 1e-11
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn(ctx.n, dtype=torch.complex128, device=dev, generator=g)
    yv = torch.randn(ctx.n, dtype=torch.complex128, device=dev, generator=g)
    Ax, Ay = torch.empty_like(x), torch.empty_like(x)
    helm.helm_spmv(A1, x, Ax)
    helm.helm_spmv(A1, yv, Ay)
    s1 = helm.helm_reduce(1, x, Ay)
    s2 = helm.helm_reduce(1, yv, Ax)
    assert abs(s1 - s2) <= 1e-12 * abs(s1)


def test_sampled_rows_at_cabin_size():
    """282,093-node cabin with its boundary data: GPU rows equal the oracle rows."""
    prob = hi.cabin_problem(100, 56, 48)
    ctx = context(prob)
    A, S, b = gpu_matrix(ctx, 100.0)
    Aref, bref = fem.system(prob, 100.0)
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.choice(ctx.n, 2000, replace=False), prob.dir_nodes[:20],
                           np.arange(0, (prob.mesh.nx + 1) * (prob.mesh.ny + 1), 97)])  # floor rows
    D = (S[rows] - Aref[rows])
    assert abs(D).max() <= 1e-14 * abs(Aref).max()
    assert np.max(np.abs(b - bref)) <= 1e-14 * np.max(np.abs(bref))


def test_fp64_fma_probe():
    # the library's FP64 FMA probe gives a finite, plausible rate (GB300: about 0.6e12 FMA/s)
    # and rejects bad arguments
    rate = helm.helm_probe_fp64_fma(2000)
    assert 1e10 < rate < 1e14
    out = helm.ctypes.c_double()
    assert helm.LIB.helm_probe_fp64_fma(0, helm.ctypes.byref(out), None) == helm.HELM_ERR_ARG
