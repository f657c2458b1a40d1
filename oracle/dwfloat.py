"""Double-word ("double-float") arithmetic in numpy float32, and the inner COCG of the
mixed-precision solve carried out in it (oracle; test infrastructure).

The benchmark's solver refines an FP64 solution with an inner COCG whose matrix, vectors,
products and updates are double-word values: unevaluated sums hi + lo of two float32 numbers,
about 48 significand bits. Its Krylov step count is decided by that arithmetic, so the oracle
that states the count runs the same arithmetic: every operation below is a correctly rounded
float32 operation (numpy float32), in the order of the published algorithms it follows:
  TwoSum        -- Knuth, TAOCP vol. 2, Sec. 4.2.2: s = fl(a + b), e = a + b - s exactly.
  FastTwoSum    -- Dekker (1971): the same in three operations when |a| >= |b|.
  TwoProd       -- with a fused multiply-add: p = fl(a b), e = fma(a, b, -p) = a b - p exactly.
  Dot2          -- Ogita, Rump & Oishi, "Accurate sum and dot product" (2005): the running sum is
                   carried with TwoSum, the rounding errors (here also the cross products
                   ah xl + al xh of double-word operands; al xl is below the format's precision)
                   go into a second float32 accumulator.
A fused multiply-add is evaluated as fl32(fl64(a b + c)): a b of two float32 numbers is exact in
float64; the float64 addition can round, so in rare cases the result is off by one float32 ulp
from a fused operation (never for TwoProd's error term, which is exactly representable).

The sparse product follows the lattice's 27-point stencil slot by slot (slot k = (di + 1) +
3 (dj + 1) + 9 (dl + 1)): three accumulators per component, one per stencil line dj, each taking
its 9 terms plane by plane (dl = -1, 0, 1; di = -1, 0, 1 within a plane), then combined as
acc[0] + acc[1] + acc[2]; the imaginary matrix parts, non-zero only next to admittance walls,
are accumulated in a second pass (slots in order) and added. Dot products of double-word vectors
are the exactly rounded sums of the products of their (exact) float64 values.

Parity: pinned by tests/test_oracle_dwfloat.py (error-free transformations exact against
rational arithmetic, the stencil product within the Dot2 error bound of the exact product,
the inner solve's result against dense LU through the refinement).
"""
import math

import numpy as np

f32 = np.float32
f64 = np.float64


# ------------------------------------------------------------------- error-free transformations

def fma(a, b, c):
    """fl32(a b + c) for float32 arrays (a b exact in float64, then rounded to float32)."""
    return (a.astype(f64) * b.astype(f64) + c.astype(f64)).astype(f32)


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fast_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def split(v):
    """float64 -> double-word (hi = fl32(v), lo = fl32(v - hi))."""
    v = np.asarray(v, dtype=f64)
    hi = v.astype(f32)
    return hi, (v - hi.astype(f64)).astype(f32)


def join(hi, lo):
    """Exact float64 value hi + lo of a normalised double-word."""
    return hi.astype(f64) + lo.astype(f64)


class Acc:
    """Double-word accumulator s + c over arrays (elementwise)."""

    def __init__(self, s, c):
        self.s = np.array(s, dtype=f32)
        self.c = np.array(c, dtype=f32)

    @classmethod
    def zeros(cls, n):
        return cls(np.zeros(n, f32), np.zeros(n, f32))

    def mac(self, ah, al, xh, xl):
        """+= (ah + al)(xh + xl): TwoProd of the heads, cross terms into the error."""
        p = ah * xh
        ah64, xh64 = f64(ah) if np.isscalar(ah) else ah.astype(f64), xh.astype(f64)
        e = (ah64 * xh64 - p.astype(f64)).astype(f32)      # fma(ah, xh, -p): exact
        e = (ah64 * xl.astype(f64) + e).astype(f32)        # fma(ah, xl, e)
        e = ((f64(al) if np.isscalar(al) else al.astype(f64)) * xh64 + e).astype(f32)  # fma(al, xh, e)
        s2, t = two_sum(self.s, p)
        self.s = s2
        self.c = self.c + (t + e)

    def add(self, h, l):
        """+= (h + l)."""
        s2, t = two_sum(self.s, h)
        self.s = s2
        self.c = self.c + (t + l)

    def get(self):
        """Normalised (hi, lo)."""
        return fast_two_sum(self.s, self.c)


# ------------------------------------------------------------------- complex double-word vectors

class CW:
    """Complex double-word vector: four float32 arrays (re.hi, re.lo, im.hi, im.lo)."""

    def __init__(self, rh, rl, ih, il):
        self.rh, self.rl, self.ih, self.il = rh, rl, ih, il

    @classmethod
    def from_complex(cls, z):
        z = np.asarray(z, dtype=np.complex128)
        rh, rl = split(z.real)
        ih, il = split(z.imag)
        return cls(rh, rl, ih, il)

    @classmethod
    def zeros(cls, n):
        return cls(*(np.zeros(n, f32) for _ in range(4)))

    def to_complex(self):
        return join(self.rh, self.rl) + 1j * join(self.ih, self.il)

    def copy(self):
        return CW(self.rh.copy(), self.rl.copy(), self.ih.copy(), self.il.copy())


def scalar(z):
    """Complex scalar -> double-word parts (float32 numbers)."""
    rh, rl = split(np.array([complex(z).real]))
    ih, il = split(np.array([complex(z).imag]))
    return rh[0], rl[0], ih[0], il[0]


def axpy(y, a, x):
    """y + a x elementwise (a a complex scalar): re = yr + ar xr - ai xi, im = yi + ar xi + ai xr."""
    arh, arl, aih, ail = scalar(a)
    re = Acc(y.rh, y.rl)
    re.mac(arh, arl, x.rh, x.rl)
    re.mac(-aih, -ail, x.ih, x.il)
    im = Acc(y.ih, y.il)
    im.mac(arh, arl, x.ih, x.il)
    im.mac(aih, ail, x.rh, x.rl)
    rh, rl = re.get()
    ih, il = im.get()
    return CW(rh, rl, ih, il)


# ------------------------------------------------------------------- 27-point stencil product

def stencil_offsets(nx, ny):
    """Column offset of slot k = (di + 1) + 3 (dj + 1) + 9 (dl + 1) on an (nx+1) x (ny+1) x ... lattice."""
    Nx, NxNy = nx + 1, (nx + 1) * (ny + 1)
    return [(k % 3 - 1) + Nx * ((k // 3) % 3 - 1) + NxNy * (k // 9 - 1) for k in range(27)]


def slots_from_csr(A, nx, ny):
    """The 27 slot arrays (complex128 [27, n]) of a matrix with the lattice's 27-point pattern:
    slot k of row i holds A[i, i + offset_k] (zero where that column is outside the lattice or
    the entry is absent)."""
    A = A.tocsr()
    n = A.shape[0]
    off = stencil_offsets(nx, ny)
    index = {o: k for k, o in enumerate(off)}
    vals = np.zeros((27, n), dtype=np.complex128)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    d = A.indices - rows
    ks = np.array([index[int(o)] for o in d])
    vals[ks, rows] = A.data
    return vals


class StencilMatrix:
    """A slot-major matrix in double-word form: real and imaginary parts of every slot split
    into (hi, lo) float32 pairs; `cplx` marks rows with a non-zero imaginary entry."""

    def __init__(self, slots, nx, ny):
        self.n = slots.shape[1]
        self.off = stencil_offsets(nx, ny)
        self.re = [split(slots[k].real) for k in range(27)]
        self.im = [split(slots[k].imag) for k in range(27)]
        self.cplx = np.any(slots.imag != 0, axis=0)
        rows = np.arange(self.n)
        # column of slot k for every row, clamped into [0, n) (the entry there is zero)
        self.idx = [np.clip(rows + self.off[k], 0, self.n - 1) for k in range(27)]

    def _gather(self, v, k):
        return v[self.idx[k]]

    def matvec(self, x):
        """q = A x in double-word arithmetic."""
        n = self.n
        ar = [Acc.zeros(n) for _ in range(3)]
        ai = [Acc.zeros(n) for _ in range(3)]
        for dl in range(3):
            for q in range(9):
                k = q + 9 * dl
                ah, al = self.re[k]
                ar[q // 3].mac(ah, al, self._gather(x.rh, k), self._gather(x.rl, k))
                ai[q // 3].mac(ah, al, self._gather(x.ih, k), self._gather(x.il, k))
        for acc in (ar, ai):
            acc[0].add(acc[1].s, acc[1].c)
            acc[0].add(acc[2].s, acc[2].c)
        rh, rl = ar[0].get()
        ih, il = ai[0].get()
        out = CW(rh, rl, ih, il)
        if np.any(self.cplx):
            rows = np.flatnonzero(self.cplx)
            br, bi = Acc.zeros(len(rows)), Acc.zeros(len(rows))
            for k in range(27):
                bh, bl = self.im[k][0][rows], self.im[k][1][rows]
                idx = np.clip(rows + self.off[k], 0, n - 1)
                br.mac(-bh, -bl, x.ih[idx], x.il[idx])
                bi.mac(bh, bl, x.rh[idx], x.rl[idx])
            fh, fl = br.get()
            gh, gl = bi.get()
            re = Acc(out.rh[rows], out.rl[rows])
            re.add(fh, fl)
            im = Acc(out.ih[rows], out.il[rows])
            im.add(gh, gl)
            out.rh[rows], out.rl[rows] = re.get()
            out.ih[rows], out.il[rows] = im.get()
        return out


# ------------------------------------------------------------------- inner COCG in double-word

def dotu(x, y):
    """x^T y of double-word vectors: exactly rounded sum of the float64 products of their values."""
    p = x.to_complex() * y.to_complex()
    return complex(math.fsum(p.real), math.fsum(p.imag))


def make_inner(M, form="plain"):
    """An inner solve for krylov.cocg_ir: COCG on M d = s in double-word arithmetic (M a
    StencilMatrix), the same steps and stopping rule as krylov.cocg_inner; scalars (alpha, beta)
    in float64, rounded to double-word where they scale a vector. form="qrec": the steps of
    krylov.cocg_inner_qrec instead (the product taken of the residual, w = M r, and M p carried
    by q = w + beta q)."""

    def inner(s, target, inner_maxit, maxit_left, stall, nrm):
        r = CW.from_complex(s)
        d = CW.zeros(len(s))
        p = r.copy()
        rho = dotu(r, r)
        best, best_it, k, est, hist = 1.0, 0, 0, 1.0, []
        if form == "qrec":
            q = M.matvec(p)
        while True:
            if form != "qrec":
                q = M.matvec(p)
            k += 1
            mu = dotu(p, q)
            if mu == 0 or rho == 0:
                return d.to_complex(), k, est, True, hist
            alpha = rho / mu
            d = axpy(d, alpha, p)
            r = axpy(r, -alpha, q)
            est = nrm(r.to_complex())
            hist.append(est)
            if est < 0.5 * best:
                best, best_it = est, k
            if est <= target or k >= inner_maxit or k >= maxit_left or (stall and k - best_it >= stall):
                return d.to_complex(), k, est, False, hist
            rho_new = dotu(r, r)
            if form == "qrec":
                w = M.matvec(r)
                beta = rho_new / rho
                p = axpy(r, beta, p)
                q = axpy(w, beta, q)
            else:
                p = axpy(r, rho_new / rho, p)
            rho = rho_new

    return inner
