"""Krylov solvers for the complex FE Helmholtz system (oracle; test infrastructure).

Paper Sec. 4 solves the complex double-precision acoustic system with Krylov methods
(after Saad, "Iterative Methods for Sparse Linear Systems"). The oracle states, step
by step in complex128 numpy, the two iterations the GPU path runs:

* ``gmres``: restarted GMRES(m), x0 = 0, right preconditioning x = M^-1 u, Arnoldi with
  classical Gram-Schmidt applied twice ("cgs2", default) or modified Gram-Schmidt
  ("mgs"), complex Givens rotations on the Hessenberg matrix (Saad 2nd ed. Sec. 6.5),
  residual estimate |g_{j+1}| checked every step; at the end of a cycle x += M^-1 V y and
  the true residual ||b - A x|| decides convergence or restart.
  Givens reading: a = h_jj, b = h_{j+1,j} (real >= 0), r = sqrt(|a|^2 + b^2),
  c = |a|/r, s = (a/|a|) b/r; c = 0, s = 1 when a = 0. Rotation (x, y) ->
  (c x + s y, -conj(s) x + c y).
* ``cocg``: conjugate orthogonal CG (van der Vorst & Melissen 1990) for complex-symmetric
  A: CG with the unconjugated bilinear form x^T y. Stop when ||r_rec||/||b|| <= tol, then
  the true residual is checked; if it misses tol the iteration restarts from the current
  x with r = b - A x. Optional stagnation rule (``stall``): when the estimate has not halved
  its best value within ``stall`` steps, the check-and-restart is taken from the iterate saved
  at the last halving of the best estimate, if that halving happened in the current run and the
  current estimate is above it (COCG's residual on near-resonant systems can grow by orders of
  magnitude; the current iterate is then far worse than an earlier one), else from the current
  iterate. The same rule picks the iterate checked when the step cap ends the iteration.

* ``bicgstab``: BiCGSTAB (van der Vorst 1992), the paper's own Sec. 4 solver (Table 3,
  "P-BiCGSTAB"; the paper does not name its preconditioner "P", so none is applied), complex
  form with Hermitian inner products (u, v) = v^H u and shadow residual r0* = r0:
  alpha = (r, r0*)/(A p, r0*), s = r - alpha A p, omega = (A s, s)/(A s, A s),
  x += alpha p + omega s, r = s - omega A s, beta = (r_new, r0*)/(r, r0*) * alpha/omega,
  p = r + beta (p - omega A p); stop on ||r||/||b|| <= tol, confirm with the true residual,
  restart from x if it misses. One iteration = two products with A.

* ``tfqmr``: transpose-free QMR (Freund 1993; as stated in Saad 2nd ed. Sec. 7.4.3), the
  paper's other Sec. 4 solver ("P-tfQMR"), complex form with (u, v) = v^H u and r0* = r0.
  Steps m = 0, 1, 2, ...: alpha is renewed on even steps from (r0*, v); every step updates
  w -= alpha A u, the direction d = u + (theta^2/alpha) eta d, theta = ||w||/tau,
  c = 1/sqrt(1 + theta^2), tau = tau theta c, eta = c^2 alpha, x += eta d; odd steps renew
  rho = (w, r0*), beta, u = w + beta u and v = A u + beta (A u_old + beta v). The bound
  ||r_m|| <= tau sqrt(m + 1) is the stopping estimate; then the true residual decides, and a
  miss restarts from x. Iteration count = steps m (one product with A per step on average).
* ``pcocg``: COCG with a diagonal preconditioner in the classical preconditioned-CG form
  (z = D^-1 r, rho = r^T z, p = z + beta p); in exact arithmetic its iterates equal those of COCG
  on S A S (S = D^-1/2) mapped back by x = S y, the form ``sym_jacobi`` builds -- an independent
  formulation used to cross-check that one.
* ``cocg_inner_qrec``: the inner COCG of the refinement with the product taken of the residual
  (w = A s) and A p carried by the recurrence q = w + beta q -- the same iteration in exact
  arithmetic, in the form where a parallel step needs one synchronisation point fewer; used to
  measure how far that form moves the step counts (oracle/measure_qrec.py).
* ``right_jacobi``: the "P" of the paper's P-BiCGSTAB / P-TFQMR read as Jacobi, applied on the
  right (A D^-1 y = b, x = D^-1 y, D = diag(A)), so residuals stay those of A x = b.

Iteration count = number of Krylov steps (products with A inside the iteration; the
true-residual products are not counted).

Inner products and norms are the exactly rounded sums (math.fsum) of the elementwise products,
the closest floating-point rendering of sum_i x_i y_i. (A BLAS dot accumulates in its own
blocked order; on these indefinite systems COCG's erratic residual history is sensitive enough
to that rounding to move the step count by up to ~10%.)

Pinned (tests/test_oracle_krylov.py): solutions equal dense LU (numpy.linalg.solve) on
small meshes, the discrete duct / rigid-box forced-mode solutions are reproduced to
round-off, a 1x1x1 Schwarz partition converges in one step, Givens rotations annihilate
and are unitary. Iteration counts themselves are parity-unpinned (the paper prints none
for these methods).
"""
import dataclasses
import math

import numpy as np
import scipy.sparse as sp


def dotu(x, y):
    """x^T y (unconjugated), exactly rounded sum of the rounded products."""
    p = np.asarray(x) * np.asarray(y)
    return complex(math.fsum(p.real), math.fsum(p.imag))


def dotc(x, y):
    """x^H y, exactly rounded sum of the rounded products."""
    return dotu(np.conj(x), y)


def nrm2(x):
    """||x||_2 = sqrt of the exactly rounded sum of |x_i|^2."""
    x = np.asarray(x)
    return math.sqrt(math.fsum(x.real * x.real + x.imag * x.imag))


@dataclasses.dataclass
class Stats:
    iterations: int = 0
    restarts: int = 0
    converged: bool = False
    relres: float = np.inf         # true ||b - A x|| / ||b|| at exit
    breakdown: bool = False
    history: list = dataclasses.field(default_factory=list)  # residual estimates per step


def givens(a, b):
    """Complex Givens (c real, s complex) taking (a, b) to (r e^{i arg a}, 0); b real >= 0."""
    if a == 0:
        return 0.0, 1.0 + 0.0j
    r = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    return abs(a) / r, (a / abs(a)) * (b / r)


def _rotate(c, s, x, y):
    return c * x + s * y, -np.conj(s) * x + c * y


def gmres(matvec, b, m, tol=1e-10, maxit=10000, precond=None, ortho="cgs2", x0=None):
    """Restarted right-preconditioned GMRES(m). Returns (x, Stats)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    Minv = precond if precond is not None else (lambda v: v)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    st = Stats()
    nb = nrm2(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st
    r = b - matvec(x)
    st.relres = nrm2(r) / nb
    if st.relres <= tol:
        st.converged = True
        return x, st
    while True:
        beta0 = nrm2(r)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta0
        V[0] = r / beta0
        j_end = 0
        for j in range(m):
            w = matvec(Minv(V[j]))
            st.iterations += 1
            if ortho == "cgs2":
                h = np.array([dotc(V[i], w) for i in range(j + 1)])
                w = w - V[: j + 1].T @ h
                h2 = np.array([dotc(V[i], w) for i in range(j + 1)])
                w = w - V[: j + 1].T @ h2
                h = h + h2
            else:  # modified Gram-Schmidt
                h = np.zeros(j + 1, dtype=np.complex128)
                for i in range(j + 1):
                    h[i] = dotc(V[i], w)
                    w = w - h[i] * V[i]
            hn = nrm2(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                H[i, j], H[i + 1, j] = _rotate(cs[i], sn[i], H[i, j], H[i + 1, j])
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j], H[j + 1, j] = _rotate(cs[j], sn[j], H[j, j], H[j + 1, j])
            g[j], g[j + 1] = _rotate(cs[j], sn[j], g[j], 0.0)
            est = abs(g[j + 1]) / nb
            st.history.append(est)
            j_end = j + 1
            if hn == 0:
                st.breakdown = True
            if est <= tol or hn == 0 or st.iterations >= maxit:
                break
            V[j + 1] = w / hn
        # least squares: R y = g[:j_end], R upper triangular
        y = np.zeros(j_end, dtype=np.complex128)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: j_end] @ y[i + 1:]) / H[i, i]
        x = x + Minv(V[:j_end].T @ y)
        r = b - matvec(x)
        st.relres = nrm2(r) / nb
        if st.relres <= tol:
            st.converged = True
            return x, st
        if st.iterations >= maxit or st.breakdown:
            return x, st
        st.restarts += 1


def cocg(matvec, b, tol=1e-10, maxit=100000, stall=None, weights=None):
    """COCG for complex-symmetric A. Returns (x, Stats). With ``weights`` w >= 0 every norm is
    the weighted norm sqrt(sum_i w_i |v_i|^2) (used by the symmetric Jacobi form, where the
    weights turn residuals of the scaled system back into residuals of the original one)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    st = Stats()
    if weights is not None:
        w = np.asarray(weights, dtype=np.float64)
        nrm2 = lambda v: math.sqrt(math.fsum(w * (v.real * v.real + v.imag * v.imag)))  # noqa: E731
    else:
        nrm2 = globals()["nrm2"]
    nb = nrm2(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st
    r = b.copy()
    best, best_it = 1.0, 0
    xb = x.copy()  # iterate at the last halving of the best estimate
    start_it = 0   # step count at the last (re)start
    while True:
        p = r.copy()
        rho = dotu(r, r)
        est = best
        while st.iterations < maxit:
            q = matvec(p)
            st.iterations += 1
            mu = dotu(p, q)
            if mu == 0 or rho == 0:
                st.breakdown = True
                break
            alpha = rho / mu
            x = x + alpha * p
            r = r - alpha * q
            est = nrm2(r) / nb
            st.history.append(est)
            if est < 0.5 * best:
                best, best_it = est, st.iterations
                xb = x.copy()
            if est <= tol or (stall and st.iterations - best_it >= stall):
                break
            rho_new = dotu(r, r)
            p = r + (rho_new / rho) * p
            rho = rho_new
        if est > tol and best < est and best_it > start_it and not st.breakdown:
            # stagnation or step cap above the best estimate of this run: check (and restart
            # from) the iterate saved at that estimate; without a halving since the last restart
            # the current iterate is kept (restarting from the same point would repeat the run)
            x = xb.copy()
        r = b - matvec(x)
        st.relres = nrm2(r) / nb
        if st.relres <= tol:
            st.converged = True
            return x, st
        if st.iterations >= maxit or st.breakdown:
            return x, st
        st.restarts += 1
        best, best_it = st.relres, st.iterations
        start_it = st.iterations
        xb = x.copy()


def bicgstab(matvec, b, tol=1e-10, maxit=100000):
    """BiCGSTAB for general complex A. Returns (x, Stats); Stats.iterations counts iterations
    (two products with A each)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    st = Stats()
    nb = nrm2(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st
    r = b.copy()
    while True:
        rs = r.copy()           # shadow residual r0*
        p = r.copy()
        rho = dotc(rs, r)       # (r, r0*) = r0*^H r
        while st.iterations < maxit:
            v = matvec(p)
            st.iterations += 1
            den = dotc(rs, v)
            if den == 0 or rho == 0:
                st.breakdown = True
                break
            alpha = rho / den
            s_ = r - alpha * v
            t = matvec(s_)
            tt = dotc(t, t).real
            omega = dotc(t, s_) / tt if tt != 0 else 0.0
            x = x + alpha * p + omega * s_
            r = s_ - omega * t
            est = nrm2(r) / nb
            st.history.append(est)
            if est <= tol:
                break
            if omega == 0:
                st.breakdown = True
                break
            rho_new = dotc(rs, r)
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            rho = rho_new
        r = b - matvec(x)
        st.relres = nrm2(r) / nb
        if st.relres <= tol:
            st.converged = True
            return x, st
        if st.iterations >= maxit or st.breakdown:
            return x, st
        st.restarts += 1


def tfqmr(matvec, b, tol=1e-10, maxit=100000):
    """Transpose-free QMR for general complex A. Returns (x, Stats); Stats.iterations counts
    steps m."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    st = Stats()
    nb = nrm2(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st
    r = b.copy()
    while True:
        rs = r.copy()                   # r0*
        w = r.copy()
        u = r.copy()
        v = matvec(u)
        au = v                          # A u for the current u
        d = np.zeros(n, dtype=np.complex128)
        tau = nrm2(r)
        theta, eta = 0.0, 0.0 + 0.0j
        rho = dotc(rs, r)
        alpha = 0.0 + 0.0j
        m = 0
        while st.iterations < maxit:
            if m % 2 == 0:
                den = dotc(rs, v)
                if den == 0 or rho == 0:
                    st.breakdown = True
                    break
                alpha = rho / den
                u_next = u - alpha * v
            else:
                au = matvec(u)
            st.iterations += 1
            w = w - alpha * au
            d = u + (theta * theta / alpha) * eta * d
            theta = nrm2(w) / tau
            c = 1.0 / np.sqrt(1.0 + theta * theta)
            tau = tau * theta * c
            eta = c * c * alpha
            x = x + eta * d
            est = tau * np.sqrt(m + 1.0) / nb
            st.history.append(est)
            if est <= tol:
                break
            if m % 2 == 0:
                u = u_next
                au = None
            else:
                rho_new = dotc(rs, w)
                if rho == 0:
                    st.breakdown = True
                    break
                beta = rho_new / rho
                au_old = au
                u = w + beta * u
                au = matvec(u)
                v = au + beta * (au_old + beta * v)
                rho = rho_new
            m += 1
        r = b - matvec(x)
        st.relres = nrm2(r) / nb
        if st.relres <= tol:
            st.converged = True
            return x, st
        if st.iterations >= maxit or st.breakdown:
            return x, st
        st.restarts += 1


def right_jacobi(A):
    """Right Jacobi preconditioning of a sparse matrix: returns (matvec of A D^-1, map y -> D^-1 y)."""
    d = np.asarray(A.diagonal(), dtype=np.complex128)
    return (lambda u: A @ (u / d)), (lambda y: y / d)


def sym_jacobi(A):
    """Symmetric Jacobi scaling of a complex-symmetric sparse A (the COCG reading of the paper's
    "P"): S = diag(s), s_i = 1 / sqrt(a_ii) (principal root), A_hat = S A S stays complex
    symmetric. A x = b is solved as A_hat y = S b, x = S y; residuals map back as r = S^-1 r_hat,
    so ||r||^2 = sum_i |a_ii| |r_hat_i|^2: returns (A_hat, s, w) with w_i = |a_ii| the norm
    weights that make cocg(..., weights=w) test the residual of A x = b."""
    d = np.asarray(A.diagonal(), dtype=np.complex128)
    s = 1.0 / np.sqrt(d)
    S = sp.diags(s)
    return (S @ A @ S).tocsr(), s, np.abs(d)


def pcocg(matvec, b, dinv, tol=1e-10, maxit=100000):
    """COCG preconditioned by the diagonal dinv (z = dinv * r), x0 = 0, stop on the true-system
    residual estimate ||r|| / ||b|| <= tol (no restarts). Returns (x, Stats)."""
    b = np.asarray(b, dtype=np.complex128)
    dinv = np.asarray(dinv, dtype=np.complex128)
    x = np.zeros_like(b)
    st = Stats()
    nb = nrm2(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rho = dotu(r, z)
    while st.iterations < maxit:
        q = matvec(p)
        st.iterations += 1
        mu = dotu(p, q)
        if mu == 0 or rho == 0:
            st.breakdown = True
            break
        alpha = rho / mu
        x = x + alpha * p
        r = r - alpha * q
        est = nrm2(r) / nb
        st.history.append(est)
        if est <= tol:
            break
        z = dinv * r
        rho_new = dotu(r, z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    st.relres = nrm2(b - matvec(x)) / nb
    st.converged = st.relres <= tol
    return x, st


def cocg_inner(matvec, s, target, inner_maxit, maxit_left, stall, nrm):
    """The inner solve of ``cocg_ir``: COCG on A d = s from d = 0, no restarts, in complex128.
    Stops when the residual estimate nrm(s_k) reaches `target`, after inner_maxit or maxit_left
    steps, on a breakdown, or after `stall` steps without a halving of its best estimate.
    Returns (d, steps, final estimate, breakdown, estimate history)."""
    d = np.zeros_like(s)
    p = s.copy()
    rho = dotu(s, s)
    best, best_it, k, est, hist = 1.0, 0, 0, 1.0, []
    while True:
        q = matvec(p)
        k += 1
        mu = dotu(p, q)
        if mu == 0 or rho == 0:
            return d, k, est, True, hist
        alpha = rho / mu
        d = d + alpha * p
        s = s - alpha * q
        est = nrm(s)
        hist.append(est)
        if est < 0.5 * best:
            best, best_it = est, k
        if est <= target or k >= inner_maxit or k >= maxit_left or (stall and k - best_it >= stall):
            return d, k, est, False, hist
        rho_new = dotu(s, s)
        p = s + (rho_new / rho) * p
        rho = rho_new


def cocg_inner_qrec(matvec, s, target, inner_maxit, maxit_left, stall, nrm):
    """``cocg_inner`` with the product taken of the residual: each step forms w = A s and gets
    A p from the recurrence q = w + beta q alongside p = s + beta p, so q = A p in exact
    arithmetic and drifts from it by rounding in floating point. In this form one pass over the
    rows can take the product and update both directions, i.e. a parallel step needs one global
    synchronisation point fewer. Same stopping rules and results as ``cocg_inner``."""
    d = np.zeros_like(s)
    p = s.copy()
    q = matvec(p)
    rho = dotu(s, s)
    best, best_it, k, est, hist = 1.0, 0, 0, 1.0, []
    while True:
        k += 1
        mu = dotu(p, q)
        if mu == 0 or rho == 0:
            return d, k, est, True, hist
        alpha = rho / mu
        d = d + alpha * p
        s = s - alpha * q
        est = nrm(s)
        hist.append(est)
        if est < 0.5 * best:
            best, best_it = est, k
        if est <= target or k >= inner_maxit or k >= maxit_left or (stall and k - best_it >= stall):
            return d, k, est, False, hist
        rho_new = dotu(s, s)
        beta = rho_new / rho
        w = matvec(s)
        p = s + beta * p
        q = w + beta * q
        rho = rho_new


def cocg_ir(matvec, b, tol=1e-10, inner_tol=1e-12, inner_maxit=100000, max_outer=20, maxit=100000, stall=None,
            weights=None, inner=None):
    """Iterative refinement around an inner COCG, all in complex128: the outer loop of the
    mixed-precision solves, stated with an FP64 inner solve. Returns (x, Stats, outer) where
    Stats.iterations counts inner COCG steps and ``outer`` the refinement steps (negative when
    the refinement stalled and the system was solved by plain COCG from zero instead).

    Outer step: r = b - A x; stop when ||r|| / ||b|| <= tol (true residual), or after max_outer
    steps or maxit inner steps; if a refinement step did not halve the residual of the previous
    one, fall back to ``cocg`` from x = 0 for the rest of the budget. Otherwise solve A d = r / ||r||
    by COCG from d = 0 (no restarts) until its residual estimate reaches
    max(inner_tol, tol ||b|| / (2 ||r||)) -- so one inner solve can reach the outer target with a
    margin of two -- or inner_maxit / maxit steps, a breakdown, or ``stall`` steps without a
    halving of its best estimate; then x += ||r|| d, unless the inner solve did not reduce its
    residual at all (estimate >= 1), in which case the correction is dropped. Norms are weighted
    by ``weights`` as in ``cocg``. ``inner`` replaces the FP64 inner solve (``cocg_inner``'s
    signature and results), e.g. by one in another arithmetic.
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    if weights is not None:
        w = np.asarray(weights, dtype=np.float64)
        nrm = lambda v: math.sqrt(math.fsum(w * (v.real * v.real + v.imag * v.imag)))  # noqa: E731
    else:
        nrm = nrm2
    solve_inner = inner if inner is not None else (lambda s_, t_, im_, ml_, st_, nm_: cocg_inner(
        matvec, s_, t_, im_, ml_, st_, nm_))
    x = np.zeros(n, dtype=np.complex128)
    st = Stats()
    outer = 0
    nb = nrm(b)
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st, outer
    prev = 1.0
    while True:
        r = b - matvec(x)
        rel = nrm(r) / nb
        st.relres = rel
        if rel <= tol:
            st.converged = True
            return x, st, outer
        if outer >= max_outer or st.iterations >= maxit:
            return x, st, outer
        if outer >= 1 and rel > 0.5 * prev:
            x, st2 = cocg(matvec, b, tol=tol, maxit=maxit - st.iterations, stall=stall, weights=weights)
            st.iterations += st2.iterations
            st.restarts += st2.restarts
            st.converged, st.relres, st.breakdown = st2.converged, st2.relres, st2.breakdown
            st.history += st2.history
            return x, st, -outer
        prev = rel
        rn = rel * nb
        outer += 1
        target = max(inner_tol, 0.5 * tol * nb / rn)
        d, k, est, bd, hist = solve_inner(r / rn, target, inner_maxit, maxit - st.iterations, stall, nrm)
        st.iterations += k
        st.breakdown = st.breakdown or bd
        st.history += [h * rel for h in hist]
        if est < 1.0:
            x = x + rn * d


def gmres_inner_c64(matvec32, s, m, target, maxit_left):
    """Inner solve of the complex64 GMRES-IR form: restarted GMRES(m) on A d = s with the
    Arnoldi basis and the products with A in complex64 (``matvec32``: a complex64 matrix times a
    complex64 vector, FP32 accumulation), the Gram-Schmidt inner products and norms accumulated
    in FP64 from the complex64 values (CGS2), the Givens rotations and the least-squares solve
    in FP64 (Saad 2nd ed. Sec. 6.5, the rotations of ``gmres``), the correction d accumulated in
    FP64. Each restart begins from the inner residual s - A d evaluated in complex64. Stops when
    the Givens estimate |g_{j+1}| / ||s|| reaches `target` or after `maxit_left` steps.
    Returns (d, steps, final estimate, breakdown, estimate history)."""
    s = np.asarray(s, dtype=np.complex128)
    n = s.shape[0]
    ns = np.linalg.norm(s)
    d = np.zeros(n, dtype=np.complex128)
    r = s.astype(np.complex64)
    k, est, hist = 0, 1.0, []
    while True:
        beta0 = np.linalg.norm(r.astype(np.complex128))
        if beta0 == 0:
            return d, k, 0.0, False, hist
        V = np.zeros((m + 1, n), dtype=np.complex64)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta0
        V[0] = (r.astype(np.complex128) / beta0).astype(np.complex64)
        j_end, bd = 0, False
        for j in range(m):
            w = matvec32(V[j]).astype(np.complex128)
            k += 1
            Vj = V[: j + 1].astype(np.complex128)
            h = Vj.conj() @ w
            w = w - Vj.T @ h
            h2 = Vj.conj() @ w
            w = w - Vj.T @ h2
            h = h + h2
            w32 = w.astype(np.complex64)
            hn = np.linalg.norm(w32.astype(np.complex128))
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                H[i, j], H[i + 1, j] = _rotate(cs[i], sn[i], H[i, j], H[i + 1, j])
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j], H[j + 1, j] = _rotate(cs[j], sn[j], H[j, j], H[j + 1, j])
            g[j], g[j + 1] = _rotate(cs[j], sn[j], g[j], 0.0)
            est = abs(g[j + 1]) / ns
            hist.append(est)
            j_end = j + 1
            bd = hn == 0
            if est <= target or bd or k >= maxit_left:
                break
            V[j + 1] = (w32.astype(np.complex128) / hn).astype(np.complex64)
        y = np.zeros(j_end, dtype=np.complex128)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: j_end] @ y[i + 1:]) / H[i, i]
        d = d + V[:j_end].astype(np.complex128).T @ y
        r = (s.astype(np.complex64) - matvec32(d.astype(np.complex64)))
        est = np.linalg.norm(r.astype(np.complex128)) / ns
        if est <= target or bd or k >= maxit_left:
            return d, k, est, bd, hist


def gmres_ir(matvec, matvec32, b, m=40, tol=1e-10, inner_reduction=1e-4, inner_maxit=5000, max_outer=20,
             maxit=100000):
    """FP64 iterative refinement around ``gmres_inner_c64`` (GMRES-IR with a complex64 inner
    solve, after Carson & Higham 2018): r = b - A x in FP64, inner GMRES(m) on A d = r / ||r||
    to an inner reduction `inner_reduction` (or the outer target, whichever is larger), x +=
    ||r|| d in FP64; stop at true rel-res <= tol, after max_outer refinement steps or maxit inner
    steps. Returns (x, Stats, outer, per-step list of (inner steps, true rel-res))."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    st = Stats()
    nb = nrm2(b)
    log, outer = [], 0
    if nb == 0:
        st.converged, st.relres = True, 0.0
        return x, st, outer, log
    while True:
        r = b - matvec(x)
        rel = nrm2(r) / nb
        st.relres = rel
        if rel <= tol:
            st.converged = True
            return x, st, outer, log
        if outer >= max_outer or st.iterations >= maxit:
            return x, st, outer, log
        outer += 1
        rn = rel * nb
        target = max(inner_reduction, 0.5 * tol * nb / rn)
        d, k, est, bd, hist = gmres_inner_c64(matvec32, r / rn, m, target, min(inner_maxit, maxit - st.iterations))
        st.iterations += k
        st.history += [h * rel for h in hist]
        x = x + rn * d
        log.append((k, float(nrm2(b - matvec(x)) / nb)))
