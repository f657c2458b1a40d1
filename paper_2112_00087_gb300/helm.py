"""Thin ctypes binding of libhelm.so (include/helm.h). Argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only converts torch CUDA
tensors to raw pointers, passes the current CUDA stream and raises on a non-OK status. If the
shared library is missing the import fails with an error naming the build command -- there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libhelm.so")

HELM_OK, HELM_ERR_ARG, HELM_ERR_CUDA, HELM_ERR_OOM, HELM_NOT_CONVERGED = 0, 1, 2, 3, 4
HELM_BREAKDOWN, HELM_NAN, HELM_PIVOT, HELM_TIMEOUT, HELM_ERR_STATE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
                6: "NAN", 7: "PIVOT", 8: "TIMEOUT", 9: "ERR_STATE"}
HELM_C128, HELM_C64 = 0, 1
HELM_FMT_CSR, HELM_FMT_DIA27 = 0, 1
HELM_SOLVER_GMRES, HELM_SOLVER_COCG, HELM_SOLVER_BICGSTAB, HELM_SOLVER_TFQMR = 0, 1, 2, 3
HELM_PRECOND_NONE, HELM_PRECOND_RAS, HELM_PRECOND_JACOBI, HELM_PRECOND_ORAS, HELM_PRECOND_ORAS2 = 0, 1, 2, 3, 4

# Symbols declared in include/helm.h (tests check the library exports all of them).
EXPORTED = ["helm_last_error", "helm_create", "helm_destroy", "helm_set_boundary", "helm_sizes",
            "helm_assemble", "helm_matrix_free", "helm_matrix_csr", "helm_matrix_dia27", "helm_spmv", "helm_reduce",
            "helm_solve", "helm_solve_batch", "helm_adjoint_grad", "helm_adjoint_seed", "helm_last_profile",
            "helm_reduce_noalloc", "helm_assemble_shared", "helm_shared_free", "helm_spmv_multi",
            "helm_probe_fp64_fma", "helm_spmv_multi_interleaved"]


class HelmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double)]


class Phys(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("rho", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("restart", ctypes.c_int32), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int32), ("precond", ctypes.c_int32), ("ras_parts", ctypes.c_int32 * 3),
                ("ras_overlap", ctypes.c_int32), ("mixed", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("stall_window", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("robin_lo", ctypes.c_double * 2), ("robin_hi", ctypes.c_double * 2)]


class Profile(ctypes.Structure):
    _fields_ = [("assemble_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("grid_blocks", ctypes.c_int32), ("ntiles", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("relres", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("iterations_c64", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libhelm.so not built (%s); run `python -m paper_2112_00087_gb300.build` "
                          "(or __graft_entry__.build())" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "helm_last_error": (ctypes.c_char_p, []),
        "helm_create": (i32, [P(vp), P(MeshDesc), P(Phys), vp]),
        "helm_destroy": (None, [vp]),
        "helm_set_boundary": (i32, [vp, vp, vp, i32, vp]),
        "helm_sizes": (i32, [vp, P(i64), P(i64), P(i64), P(i32)]),
        "helm_assemble": (i32, [vp, d, i32, i32, P(vp), vp]),
        "helm_matrix_free": (None, [vp]),
        "helm_matrix_csr": (i32, [vp, P(i64), P(i64), P(i32), P(vp), P(vp), P(vp)]),
        "helm_matrix_dia27": (i32, [vp, P(i64), P(i32), P(vp)]),
        "helm_spmv": (i32, [vp, vp, vp, vp]),
        "helm_reduce": (i32, [i32, i64, vp, vp, P(d), vp]),
        "helm_reduce_noalloc": (i32, [i32, i64, vp, vp, P(d), vp]),
        "helm_solve": (i32, [vp, P(d), i32, P(SolveOpts), vp, P(SolveStats)]),
        "helm_solve_batch": (i32, [P(vp), P(d), i32, P(SolveOpts), P(vp), P(SolveStats)]),
        "helm_adjoint_grad": (i32, [vp, P(d), i32, P(SolveOpts), vp, vp, vp, vp, P(d)]),
        "helm_adjoint_seed": (i32, [vp, P(d), i32, P(SolveOpts), vp, vp, vp, vp]),
        "helm_last_profile": (i32, [P(Profile)]),
        "helm_assemble_shared": (i32, [vp, i32, P(vp)]),
        "helm_shared_free": (None, [vp]),
        "helm_spmv_multi": (i32, [vp, P(d), i32, vp, vp, vp]),
        "helm_probe_fp64_fma": (i32, [i32, P(d), vp]),
        "helm_spmv_multi_interleaved": (i32, [vp, P(d), i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()
LIB_PATH = _LIB_PATH


def _check(status: int, allow=()):
    if status != HELM_OK and status not in allow:
        raise HelmError(status, LIB.helm_last_error().decode())
    return status


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_opts(solver="cocg", restart=50, tol=1e-10, maxit=100000, precond=None, ras_parts=(8, 4, 4),
              ras_overlap=2, mixed=False, inner_tol=1e-4, inner_maxit=5000, max_outer=50, stall_window=0,
              robin=None) -> SolveOpts:
    o = SolveOpts()
    o.solver = {"gmres": HELM_SOLVER_GMRES, "cocg": HELM_SOLVER_COCG, "bicgstab": HELM_SOLVER_BICGSTAB,
                "tfqmr": HELM_SOLVER_TFQMR}[solver]
    o.restart = restart
    o.tol = tol
    o.maxit = maxit
    o.precond = {None: HELM_PRECOND_NONE, "ras": HELM_PRECOND_RAS, "jacobi": HELM_PRECOND_JACOBI,
                 "oras": HELM_PRECOND_ORAS, "oras2": HELM_PRECOND_ORAS2}[precond]
    # precond "oras2": robin = (c_lo, c_hi), the dimensionless two-sided interface coefficients
    if robin is not None:
        lo, hi = complex(robin[0]), complex(robin[1])
        o.robin_lo[:] = [lo.real, lo.imag]
        o.robin_hi[:] = [hi.real, hi.imag]
    o.ras_parts[:] = list(ras_parts)
    o.ras_overlap = ras_overlap
    # mixed: False / True (complex64 inner) / "c64" / "dw" (double-word inner)
    o.mixed = {False: 0, True: 1, "c64": 1, "dw": 2}[mixed]
    o.inner_tol = inner_tol
    o.inner_maxit = inner_maxit
    o.max_outer = max_outer
    o.stall_window = stall_window
    return o


class Context:
    """helm_create / helm_set_boundary / helm_destroy around one lattice."""

    def __init__(self, nx, ny, nz, Lx, Ly, Lz, c=340.0, rho=1.2, stream=None):
        self.mesh = MeshDesc(nx, ny, nz, Lx, Ly, Lz)
        self.phys = Phys(c, rho)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(LIB.helm_create(ctypes.byref(h), ctypes.byref(self.mesh), ctypes.byref(self.phys),
                               ctypes.c_void_p(self._stream.cuda_stream)))
        self.handle = h
        n, nnz, nbf, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(LIB.helm_sizes(h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nbf), ctypes.byref(nd)))
        self.n, self.nnz, self.n_bface = n.value, nnz.value, nbf.value
        self.n_dir = 0
        self._keep = []

    def set_boundary(self, beta: Optional[torch.Tensor], dir_nodes: Optional[torch.Tensor],
                     p_dir: Optional[torch.Tensor]):
        if beta is not None:
            assert beta.dtype == torch.complex128 and beta.numel() == self.n_bface
        nd = 0 if dir_nodes is None else dir_nodes.numel()
        if nd:
            assert dir_nodes.dtype == torch.int32 and p_dir.dtype == torch.complex128 and p_dir.numel() == nd
        _check(LIB.helm_set_boundary(self.handle, _ptr(beta), _ptr(dir_nodes) if nd else None, nd,
                                     _ptr(p_dir) if nd else None))
        self.n_dir = nd
        # keep the sources alive until the stream has passed the copies
        self._keep = [beta, dir_nodes, p_dir]

    def close(self):
        if self.handle is not None and self.handle.value:
            LIB.helm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """helm_assemble result; .csr() / .dia27() copy the stored values into torch tensors."""

    def __init__(self, ctx: Context, freq: float, precision=HELM_C128, with_rhs=True, fmt=HELM_FMT_CSR):
        self.ctx = ctx
        h = ctypes.c_void_p()
        self.rhs = torch.empty(ctx.n, dtype=torch.complex128, device="cuda") if with_rhs else None
        _check(LIB.helm_assemble(ctx.handle, float(freq), precision, fmt, ctypes.byref(h), _ptr(self.rhs)))
        self.handle = h
        self.precision = precision
        self.format = fmt
        self.n, self.nnz = ctx.n, ctx.nnz

    def csr(self):
        n, nnz, prec = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        rp, cl, vl = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(LIB.helm_matrix_csr(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(prec),
                                   ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl)))
        vdt = torch.complex64 if prec.value == HELM_C64 else torch.complex128
        rowptr = torch.empty(n.value + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(nnz.value, dtype=torch.int32, device="cuda")
        val = torch.empty(nnz.value, dtype=vdt, device="cuda")
        torch.cuda.synchronize()
        _cuda_copy(rowptr, rp.value)
        _cuda_copy(col, cl.value)
        _cuda_copy(val, vl.value)
        return rowptr, col, val

    def dia27(self):
        """Complex values [27, n] (slot k = (di+1) + 3(dj+1) + 9(dl+1)) from the split layout."""
        n, prec, vl = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_void_p()
        _check(LIB.helm_matrix_dia27(self.handle, ctypes.byref(n), ctypes.byref(prec), ctypes.byref(vl)))
        real = torch.float32 if prec.value == HELM_C64 else torch.float64
        flat = torch.as_tensor(_DevView(vl.value, (54 * n.value,), "<f4" if real == torch.float32 else "<f8"),
                               device="cuda").clone()
        return torch.complex(flat[:27 * n.value], flat[27 * n.value:]).reshape(27, n.value)

    def free(self):
        if self.handle is not None and self.handle.value:
            LIB.helm_matrix_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _DevView:
    """Foreign device memory described by __cuda_array_interface__ (no ownership)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _cuda_copy(dst: torch.Tensor, src_ptr: int):
    """Copy library-owned device memory into a torch tensor of the same size and dtype."""
    if dst.dtype in (torch.complex64, torch.complex128):
        real = torch.float32 if dst.dtype == torch.complex64 else torch.float64
        view = torch.as_tensor(_DevView(src_ptr, (dst.numel(), 2), "<f4" if real == torch.float32 else "<f8"),
                               device="cuda")
        dst.copy_(torch.view_as_complex(view))
    else:
        assert dst.dtype == torch.int32
        dst.copy_(torch.as_tensor(_DevView(src_ptr, (dst.numel(),), "<i4"), device="cuda"))


# ----------------------------------------------------------------------------------------------
# Functions with the C-ABI names
# ----------------------------------------------------------------------------------------------

def helm_create(nx, ny, nz, Lx, Ly, Lz, c=340.0, rho=1.2, stream=None) -> Context:
    return Context(nx, ny, nz, Lx, Ly, Lz, c, rho, stream)


def helm_set_boundary(ctx: Context, beta, dir_nodes, p_dir):
    ctx.set_boundary(beta, dir_nodes, p_dir)


def helm_assemble(ctx: Context, freq: float, precision=HELM_C128, with_rhs=True, fmt=HELM_FMT_CSR) -> Matrix:
    return Matrix(ctx, freq, precision, with_rhs, fmt)


def helm_spmv(A: Matrix, x: torch.Tensor, y: torch.Tensor, stream=None):
    want = torch.complex64 if A.precision == HELM_C64 else torch.complex128
    assert x.dtype == want and y.dtype == want and x.numel() == A.n and y.numel() == A.n
    _check(LIB.helm_spmv(A.handle, _ptr(x), _ptr(y), _stream(stream)))


class SharedOperator:
    """helm_assemble_shared result: K, M, B of the context's lattice, for helm_spmv_multi."""

    def __init__(self, ctx: Context, precision=HELM_C128):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(LIB.helm_assemble_shared(ctx.handle, precision, ctypes.byref(h)))
        self.handle = h
        self.precision = precision
        self.n = ctx.n

    def close(self):
        if self.handle:
            LIB.helm_shared_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def helm_assemble_shared(ctx: Context, precision=HELM_C128) -> SharedOperator:
    return SharedOperator(ctx, precision)


def helm_spmv_multi(S: SharedOperator, freqs: Sequence[float], X: torch.Tensor, Y: torch.Tensor, stream=None):
    """Y[f] = A(freqs[f]) X[f]; X, Y [nfreq, n] contiguous, complex in the precision of S."""
    want = torch.complex64 if S.precision == HELM_C64 else torch.complex128
    nf = len(freqs)
    assert X.dtype == want and Y.dtype == want and X.is_contiguous() and Y.is_contiguous()
    assert X.numel() == nf * S.n and Y.numel() == nf * S.n
    fr = (ctypes.c_double * max(1, nf))(*[float(f) for f in freqs])
    _check(LIB.helm_spmv_multi(S.handle, fr, nf, _ptr(X), _ptr(Y), _stream(stream)))


def helm_spmv_multi_interleaved(S: SharedOperator, freqs: Sequence[float], X: torch.Tensor, Y: torch.Tensor,
                                stream=None):
    """Y[i, f] = (A(freqs[f]) X[:, f])_i; X, Y [n, nfreq] contiguous (node-major), complex in the
    precision of S; nfreq 2, 4, 8 (complex64) or 1, 2, 4, 8 (complex128)."""
    want = torch.complex64 if S.precision == HELM_C64 else torch.complex128
    nf = len(freqs)
    assert X.dtype == want and Y.dtype == want and X.is_contiguous() and Y.is_contiguous()
    assert X.numel() == nf * S.n and Y.numel() == nf * S.n
    fr = (ctypes.c_double * max(1, nf))(*[float(f) for f in freqs])
    _check(LIB.helm_spmv_multi_interleaved(S.handle, fr, nf, _ptr(X), _ptr(Y), _stream(stream)))


def helm_reduce(op: int, x: torch.Tensor, y: Optional[torch.Tensor] = None, stream=None) -> complex:
    assert x.dtype == torch.complex128 and (y is None or (y.dtype == torch.complex128 and y.numel() == x.numel()))
    out = (ctypes.c_double * 2)()
    _check(LIB.helm_reduce(op, x.numel(), _ptr(x), _ptr(y), out, _stream(stream)))
    return complex(out[0], out[1])


def helm_reduce_noalloc(op: int, x: torch.Tensor, y: Optional[torch.Tensor] = None, stream=None) -> complex:
    """helm_reduce without device allocation (static library scratch; n <= 16,777,216)."""
    assert x.dtype == torch.complex128 and (y is None or (y.dtype == torch.complex128 and y.numel() == x.numel()))
    out = (ctypes.c_double * 2)()
    _check(LIB.helm_reduce_noalloc(op, x.numel(), _ptr(x), _ptr(y), out, _stream(stream)))
    return complex(out[0], out[1])


def helm_solve(ctx: Context, freqs: Sequence[float], opts: SolveOpts, p_out: Optional[torch.Tensor] = None,
               raise_on_fail=True):
    """Solve every frequency; returns (p [nfreq, n] complex128 on the GPU, list of stats dicts)."""
    nf = len(freqs)
    if p_out is None:
        p_out = torch.empty((nf, ctx.n), dtype=torch.complex128, device="cuda")
    assert p_out.dtype == torch.complex128 and p_out.numel() == nf * ctx.n and p_out.is_contiguous()
    fr = (ctypes.c_double * nf)(*[float(f) for f in freqs])
    st = (SolveStats * nf)()
    status = LIB.helm_solve(ctx.handle, fr, nf, ctypes.byref(opts), _ptr(p_out), st)
    if raise_on_fail:
        _check(status)
    return p_out, [s.as_dict() for s in st]


def helm_solve_batch(ctxs: List[Context], freqs: Sequence[float], opts: SolveOpts,
                     p_outs: Optional[List[torch.Tensor]] = None, raise_on_fail=True):
    """One system per (context, frequency); all advance in one persistent launch."""
    ns = len(ctxs)
    if p_outs is None:
        p_outs = [torch.empty(c.n, dtype=torch.complex128, device="cuda") for c in ctxs]
    hs = (ctypes.c_void_p * ns)(*[c.handle.value for c in ctxs])
    ps = (ctypes.c_void_p * ns)(*[p.data_ptr() for p in p_outs])
    fr = (ctypes.c_double * ns)(*[float(f) for f in freqs])
    st = (SolveStats * ns)()
    status = LIB.helm_solve_batch(hs, fr, ns, ctypes.byref(opts), ps, st)
    if raise_on_fail:
        _check(status)
    return p_outs, [s.as_dict() for s in st]


def helm_adjoint_grad(ctx: Context, freqs: Sequence[float], opts: SolveOpts, p: torch.Tensor, w: torch.Tensor):
    """Listener objective J = sum_f sum_i w_i |p_i|^2 and its gradients (grad_beta, grad_pdir)."""
    nf = len(freqs)
    assert p.dtype == torch.complex128 and p.numel() == nf * ctx.n and w.dtype == torch.float64
    gb = torch.empty(ctx.n_bface, dtype=torch.complex128, device="cuda")
    gd = torch.empty(max(ctx.n_dir, 1), dtype=torch.complex128, device="cuda")
    J = ctypes.c_double()
    fr = (ctypes.c_double * nf)(*[float(f) for f in freqs])
    _check(LIB.helm_adjoint_grad(ctx.handle, fr, nf, ctypes.byref(opts), _ptr(p), _ptr(w), _ptr(gb), _ptr(gd),
                                 ctypes.byref(J)))
    return J.value, gb, gd[:ctx.n_dir]


def helm_adjoint_seed(ctx: Context, freqs: Sequence[float], opts: SolveOpts, p: torch.Tensor,
                      grad_p: torch.Tensor):
    nf = len(freqs)
    gb = torch.empty(ctx.n_bface, dtype=torch.complex128, device="cuda")
    gd = torch.empty(max(ctx.n_dir, 1), dtype=torch.complex128, device="cuda")
    fr = (ctypes.c_double * nf)(*[float(f) for f in freqs])
    _check(LIB.helm_adjoint_seed(ctx.handle, fr, nf, ctypes.byref(opts), _ptr(p), _ptr(grad_p.contiguous()),
                                 _ptr(gb), _ptr(gd)))
    return gb, gd[:ctx.n_dir]


def helm_last_profile() -> dict:
    pr = Profile()
    _check(LIB.helm_last_profile(ctypes.byref(pr)))
    return pr.as_dict()


def helm_probe_fp64_fma(iters: int = 20000, stream=None) -> float:
    """Measured FP64 fused multiply-add rate of the device (FMA/s)."""
    out = ctypes.c_double()
    _check(LIB.helm_probe_fp64_fma(int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


class HelmSolve(torch.autograd.Function):
    """p = solve(beta, p_dir) for every frequency, differentiable in beta and p_dir.

    forward(ctx_obj, freqs, opts, dir_nodes, beta, p_dir) -> p [nfreq, n] complex128.
    backward uses the hand-written adjoint (helm_adjoint_seed): one adjoint solve per frequency
    with the same complex-symmetric matrix, then per-quad / per-Dirichlet-node gradient kernels.
    """

    @staticmethod
    def forward(fctx, hctx: Context, freqs, opts: SolveOpts, dir_nodes, beta, p_dir):
        hctx.set_boundary(beta.detach().contiguous(), dir_nodes, p_dir.detach().contiguous())
        p, _ = helm_solve(hctx, freqs, opts)
        fctx.hctx, fctx.freqs, fctx.opts = hctx, list(freqs), opts
        fctx.save_for_backward(p)
        return p

    @staticmethod
    def backward(fctx, grad_p):
        (p,) = fctx.saved_tensors
        gb, gd = helm_adjoint_seed(fctx.hctx, fctx.freqs, fctx.opts, p, grad_p.contiguous())
        return None, None, None, None, gb, gd
