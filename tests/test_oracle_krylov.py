"""Pins of the oracle's Krylov solvers and Schwarz preconditioner (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import helm_inputs as hi
from oracle import fem, krylov, ras


def test_givens_annihilates_and_is_unitary():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.standard_normal() + 1j * rng.standard_normal()
        b = abs(rng.standard_normal())
        c, s = krylov.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-15 * abs(a)
        assert np.allclose(G.conj().T @ G, np.eye(2), atol=1e-15)
        assert abs(abs(out[0]) - np.hypot(abs(a), b)) < 1e-14
    c, s = krylov.givens(0.0, 2.0)
    assert c == 0 and s == 1


@pytest.mark.parametrize("ortho", ["cgs2", "mgs"])
def test_gmres_diagonal_converges_in_n_steps(ortho):
    # Krylov space of a diagonal matrix with 6 distinct eigenvalues and a generic rhs has
    # dimension 6: full GMRES terminates at step 6 with the exact solution
    d = np.array([1.0, 2.0 + 1j, -3.0, 0.5j + 4, 7.0, -1.0 - 2j])
    A = sp.diags(d)
    b = np.arange(1, 7) + 0.5j
    x, st = krylov.gmres(lambda v: A @ v, b, m=20, tol=1e-14)
    assert st.converged and st.iterations <= 6
    assert np.allclose(x, b / d, rtol=1e-13, atol=0)


def test_cocg_real_spd_is_cg():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((8, 8))
    A = Q @ Q.T + 8 * np.eye(8)
    b = rng.standard_normal(8) + 0j
    x, st = krylov.cocg(lambda v: A @ v, b, tol=1e-13)
    assert st.converged and st.iterations <= 12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11)


@pytest.mark.parametrize("dims,f", [((3, 2, 2), 150.0), ((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_solvers_match_dense_lu_small(dims, f):
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    mv = lambda v: A @ v
    for x, st in (krylov.gmres(mv, b, 30, tol=1e-12), krylov.gmres(mv, b, 30, tol=1e-12, ortho="mgs"),
                  krylov.cocg(mv, b, tol=1e-12)):
        assert st.converged
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_solvers_match_sparse_lu_on_box100():
    # at rel-res 1e-10 the forward error is bounded by cond(A) * 1e-10 (about 5e-8 here), so the
    # value pin runs to 1e-13 and the 1e-10 runs are checked by their true residual
    w = hi.workload("box100")
    A, b = fem.system(w.problems[0], 100.0)
    ref = spl.spsolve(A.tocsc(), b)
    mv = lambda v: A @ v
    x, st = krylov.gmres(mv, b, 30, tol=1e-13)
    assert st.converged and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    x2, st2 = krylov.cocg(mv, b, tol=1e-13)
    assert st2.converged and np.linalg.norm(x2 - ref) <= 1e-9 * np.linalg.norm(ref)
    _, st = krylov.gmres(mv, b, 30, tol=1e-10)
    _, st2 = krylov.cocg(mv, b, tol=1e-10)
    assert st.converged and st.relres <= 1e-10 and st2.converged and st2.relres <= 1e-10
    # CGS2 and MGS run the same Krylov iteration: counts agree within 5%
    _, st3 = krylov.gmres(mv, b, 30, tol=1e-10, ortho="mgs")
    assert abs(st3.iterations - st.iterations) <= 0.05 * st.iterations


def test_gmres_reproduces_forced_rigid_box_mode():
    # rigid box, no Dirichlet: (K - k^2 M) p = M v with v a tensor cosine has p = v/(lam_h - k^2)
    mesh = hi.Mesh(6, 5, 4, 1.0, 0.8, 0.6)
    K, M = fem.assemble_KM(mesh)
    k = 2 * np.pi * 120.0 / hi.C_SOUND
    A = (K - k * k * M).astype(np.complex128)
    i = np.arange(7)[None, None, :]
    j = np.arange(6)[None, :, None]
    l = np.arange(5)[:, None, None]
    v = (np.cos(np.pi * 2 * i / 6) * np.cos(np.pi * 1 * j / 5) * np.cos(np.pi * 1 * l / 4)).ravel()
    th = lambda a, n, h: (6 / h ** 2) * (1 - np.cos(np.pi * a / n)) / (2 + np.cos(np.pi * a / n))
    lam = th(2, 6, 1 / 6) + th(1, 5, 0.16) + th(1, 4, 0.15)
    x, st = krylov.gmres(lambda u: A @ u, M @ v + 0j, 40, tol=1e-13)
    assert st.converged
    assert np.linalg.norm(x - v / (lam - k * k)) <= 1e-11 * np.linalg.norm(v / (lam - k * k))


def test_ras_single_block_is_exact_inverse():
    prob = hi.small_box_problem(6, 5, 4)
    A, b = fem.system(prob, 150.0)
    P = ras.RAS(A, prob.mesh, parts=(1, 1, 1), overlap=2)
    x, st = krylov.gmres(lambda v: A @ v, b, 10, tol=1e-12, precond=P)
    assert st.converged and st.iterations == 1


def test_ras_partition_covers_every_node_once():
    mesh = hi.Mesh(100, 56, 48, *hi.CABIN)
    subs = ras.subdomains(mesh, (8, 4, 4), 2)
    own = np.zeros((101, 57, 49), dtype=int)
    for (o, e) in subs:
        own[o[0][0]:o[0][1], o[1][0]:o[1][1], o[2][0]:o[2][1]] += 1
        for (lo, hi_), (elo, ehi) in zip(o, e):
            assert elo == max(0, lo - 2) and ehi <= hi_ + 2
    assert own.min() == 1 and own.max() == 1
    assert len(subs) == 128


def test_ras_gmres_solution_equals_direct():
    prob = hi.small_box_problem(12, 10, 8)
    A, b = fem.system(prob, 200.0)
    P = ras.RAS(A, prob.mesh, parts=(3, 2, 2), overlap=2)
    x, st = krylov.gmres(lambda v: A @ v, b, 30, tol=1e-11, precond=P)
    ref = spl.spsolve(A.tocsc(), b)
    assert st.converged
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    _, st0 = krylov.gmres(lambda v: A @ v, b, 30, tol=1e-11)
    assert st.iterations < st0.iterations


def test_cocg_stagnation_restart_reaches_the_same_solution():
    # a restarted COCG (short stagnation window, so it restarts many times) still converges to the
    # dense-LU solution; the restarts are counted
    prob = hi.small_box_problem(6, 4, 3)
    A, b = fem.system(prob, 230.0)
    ref = np.linalg.solve(A.toarray(), b)
    x, st = krylov.cocg(lambda v: A @ v, b, tol=1e-12, maxit=20000, stall=20)
    assert st.converged and st.restarts > 0
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,f", [((3, 2, 2), 150.0), ((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_bicgstab_matches_dense_lu(dims, f):
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    x, st = krylov.bicgstab(lambda v: A @ v, b, tol=1e-12)
    assert st.converged
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_bicgstab_on_nonsymmetric_system_and_real_spd():
    # BiCGSTAB needs no symmetry: a random complex nonsymmetric, diagonally dominant system
    rng = np.random.default_rng(2)
    n = 30
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 12 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, st = krylov.bicgstab(lambda v: A @ v, b, tol=1e-13)
    assert st.converged and np.allclose(x, np.linalg.solve(A, b), rtol=1e-11)
    # on a 1x1 system it converges in one iteration
    x1, st1 = krylov.bicgstab(lambda v: 3.0 * v, np.array([2.0 + 1j]), tol=1e-14)
    assert st1.converged and st1.iterations == 1 and abs(x1[0] - (2.0 + 1j) / 3.0) < 1e-15


@pytest.mark.parametrize("dims,f", [((3, 2, 2), 150.0), ((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_jacobi_tfqmr_and_bicgstab_match_dense_lu(dims, f):
    # P-TFQMR / P-BiCGSTAB with the Jacobi reading of "P", right-preconditioned
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    mv, unscale = krylov.right_jacobi(A)
    for solver in (krylov.tfqmr, krylov.bicgstab):
        y, st = solver(mv, b, tol=1e-12, maxit=20000)
        assert st.converged, solver.__name__
        assert np.linalg.norm(unscale(y) - ref) <= 1e-9 * np.linalg.norm(ref)
        # right preconditioning: the residual of A D^-1 y = b is the residual of A x = b
        assert np.linalg.norm(b - A @ unscale(y)) <= 1e-12 * np.linalg.norm(b) * 1.01


def test_tfqmr_quasi_residual_bounds_the_true_residual():
    # ||b - A x_m|| <= tau_m sqrt(m + 1) at every step (Freund's bound): x_m after exactly m steps
    # against the estimate the iteration reports for step m; a wrong tau / eta / d recurrence
    # breaks it within a few steps
    rng = np.random.default_rng(4)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 9 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for k in range(1, 25):
        x, st = krylov.tfqmr(lambda v: A @ v, b, tol=1e-300, maxit=k)
        assert st.iterations == k
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert true <= st.history[-1] * (1 + 1e-10), (k, true, st.history[-1])
    x, st = krylov.tfqmr(lambda v: A @ v, b, tol=1e-13)
    assert st.converged and np.allclose(x, np.linalg.solve(A, b), rtol=1e-11)


def test_tfqmr_one_by_one_and_zero_rhs():
    x, st = krylov.tfqmr(lambda v: 3.0 * v, np.array([2.0 + 1j]), tol=1e-14)
    assert st.converged and abs(x[0] - (2.0 + 1j) / 3.0) < 1e-15
    x, st = krylov.tfqmr(lambda v: 3.0 * v, np.zeros(4, dtype=complex))
    assert st.converged and st.iterations == 0 and not x.any()


@pytest.mark.parametrize("dims,f", [((3, 2, 2), 150.0), ((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_sym_jacobi_cocg_matches_dense_lu(dims, f):
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    Ah, s, w = krylov.sym_jacobi(A)
    # the scaled matrix stays complex symmetric (to rounding of the two products)
    assert abs(Ah - Ah.T).max() <= 1e-15 * abs(Ah).max()
    y, st = krylov.cocg(lambda v: Ah @ v, s * b, tol=1e-12, weights=w)
    x = s * y
    assert st.converged
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # the weighted residual the iteration reports is the residual of the original system (to
    # the rounding of a residual computed near 1e-13, about 1e-16 ||A|| ||x|| / ||b||)
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(st.relres - true) <= 1e-6 * true + 1e-15
    # and its weighted right-hand-side norm is ||b||
    assert abs(np.sqrt(np.sum(w * np.abs(s * b) ** 2)) - np.linalg.norm(b)) <= 1e-14 * np.linalg.norm(b)


def test_weighted_norm_cocg_with_unit_weights_is_plain_cocg():
    prob = hi.small_box_problem(6, 4, 3)
    A, b = fem.system(prob, 230.0)
    x1, s1 = krylov.cocg(lambda v: A @ v, b, tol=1e-10)
    x2, s2 = krylov.cocg(lambda v: A @ v, b, tol=1e-10, weights=np.ones(len(b)))
    assert s1.iterations == s2.iterations and np.array_equal(x1, x2)


def test_sym_jacobi_form_equals_preconditioned_cocg():
    # two formulations of Jacobi-preconditioned COCG: S A S with weighted norms (what the GPU
    # runs) and classical preconditioned COCG with z = D^-1 r. Same iterates up to rounding and
    # the same residual history, step by step.
    prob = hi.small_box_problem(10, 8, 6)
    A, b = fem.system(prob, 150.0)
    Ah, s, w = krylov.sym_jacobi(A)
    dinv = 1.0 / A.diagonal()
    for k in (1, 2, 5):
        y, st1 = krylov.cocg(lambda v: Ah @ v, s * b, tol=1e-300, maxit=k, weights=w)
        x, st2 = krylov.pcocg(lambda v: A @ v, b, dinv, tol=1e-300, maxit=k)
        assert np.linalg.norm(s * y - x) <= 1e-11 * np.linalg.norm(x)
    # later iterates drift apart along ill-conditioned directions (1e-2 at step 20 here) while the
    # residual histories, which both forms measure on A x = b, still agree to rounding
    _, st1 = krylov.cocg(lambda v: Ah @ v, s * b, tol=1e-300, maxit=40, weights=w)
    _, st2 = krylov.pcocg(lambda v: A @ v, b, dinv, tol=1e-300, maxit=40)
    assert np.allclose(st1.history, st2.history, rtol=1e-8, atol=0)
    _, st1 = krylov.cocg(lambda v: Ah @ v, s * b, tol=1e-10, weights=w)
    _, st2 = krylov.pcocg(lambda v: A @ v, b, dinv, tol=1e-10)
    assert abs(st1.iterations - st2.iterations) <= 1 and st2.converged


@pytest.mark.parametrize("dims,f", [((3, 2, 2), 150.0), ((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_refined_cocg_matches_dense_lu(dims, f):
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    Ah, s, w = krylov.sym_jacobi(A)
    y, st, outer = krylov.cocg_ir(lambda v: Ah @ v, s * b, tol=1e-12, weights=w)
    x = s * y
    assert st.converged and outer >= 1
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


def test_refined_cocg_first_inner_solve_is_cocg_to_half_the_tolerance():
    # In FP64 the first inner solve (from d = 0 on r / ||r|| = b / ||b||) is COCG on b up to a
    # scaling of every vector by 1 / ||b||; with the inner target tol / 2 it takes the steps plain
    # COCG takes to reach tol / 2, and its result already meets tol, so one refinement step ends.
    for dims, f in (((10, 8, 6), 100.0), ((13, 7, 5), 230.0)):
        prob = hi.small_box_problem(*dims)
        A, b = fem.system(prob, f)
        Ah, s, w = krylov.sym_jacobi(A)
        mv = lambda v: Ah @ v
        _, st_ir, outer = krylov.cocg_ir(mv, s * b, tol=1e-10, weights=w)
        _, st_c = krylov.cocg(mv, s * b, tol=0.5e-10, weights=w)
        assert outer == 1 and st_ir.converged
        assert abs(st_ir.iterations - st_c.iterations) <= 1, (st_ir.iterations, st_c.iterations)
        # same residual history step by step (rounding of the 1 / ||b|| scaling only)
        # (the erratic history amplifies rounding later on)
        assert np.allclose(st_ir.history[:20], st_c.history[:20], rtol=1e-9, atol=0)


def test_refined_cocg_outer_residual_is_the_inner_estimate():
    # with an FP64 inner solve the correction is applied exactly (up to rounding): after each
    # refinement step the true relative residual equals the inner solve's final estimate times
    # the relative residual it started from; capped inner solves need several refinement steps
    prob = hi.small_box_problem(6, 4, 3)
    A, b = fem.system(prob, 10.0)
    prev = 1.0
    for mo in (1, 2, 3):
        _, st, outer = krylov.cocg_ir(lambda v: A @ v, b, tol=1e-12, inner_maxit=8, max_outer=mo)
        assert outer == mo and st.iterations == 8 * mo and not st.converged
        assert abs(st.relres - st.history[-1]) <= 1e-9 * st.relres  # history holds est * rel_start
        assert st.relres < 0.5 * prev
        prev = st.relres


def test_refined_cocg_falls_back_to_cocg_when_refinement_stalls():
    # the fourth capped inner solve of this system does not reduce its residual: the correction
    # is dropped, the refinement stalls and hands the system to plain COCG from zero, whose
    # result it returns unchanged
    prob = hi.small_box_problem(6, 4, 3)
    A, b = fem.system(prob, 10.0)
    x, st, outer = krylov.cocg_ir(lambda v: A @ v, b, tol=1e-12, inner_maxit=8)
    xc, stc = krylov.cocg(lambda v: A @ v, b, tol=1e-12)
    assert outer == -4 and st.converged
    assert st.iterations == 32 + stc.iterations
    assert np.array_equal(x, xc)


@pytest.mark.parametrize("dims,f", [((6, 4, 3), 230.0), ((10, 8, 6), 100.0)])
def test_gmres_ir_complex64_inner_matches_dense_lu(dims, f):
    # FP64 refinement around a complex64 inner GMRES(40) reaches the FP64 solution: each
    # refinement step multiplies the FP64 residual by about the inner reduction
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    A32 = A.astype(np.complex64)
    x, st, outer, log = krylov.gmres_ir(lambda v: A @ v, lambda v: A32 @ v, b, m=40, tol=1e-12)
    assert st.converged and outer >= 2
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    rels = [r for _, r in log]
    assert all(r2 < r1 for r1, r2 in zip(rels, rels[1:]))
    assert rels[0] <= 1e-3  # the first inner solve alone reaches the inner reduction (1e-4) to the
    #                         accuracy complex64 allows


def test_gmres_inner_complex64_stops_at_its_target():
    prob = hi.small_box_problem(6, 4, 3)
    A, b = fem.system(prob, 150.0)
    A32 = A.astype(np.complex64)
    s = b / np.linalg.norm(b)
    d, k, est, bd, hist = krylov.gmres_inner_c64(lambda v: A32 @ v, s, 40, 1e-4, 10000)
    assert est <= 1e-4 and not bd
    assert np.linalg.norm(s - A @ d) <= 2e-4  # the FP64 residual of the correction, to complex64 accuracy


def test_residual_product_form_of_the_inner_cocg():
    # cocg_inner_qrec is cocg_inner with A p carried by a recurrence: the same iteration in
    # exact arithmetic, so the first residual estimates agree to rounding (a wrong recurrence --
    # q = w + beta p, p = s + beta q, a missing beta -- breaks this at the second step), and
    # through the refinement it reaches the dense-LU solution
    for dims, f in (((10, 8, 6), 100.0), ((13, 7, 5), 230.0)):
        prob = hi.small_box_problem(*dims)
        A, b = fem.system(prob, f)
        Ah, s, w = krylov.sym_jacobi(A)
        mv = lambda v: Ah @ v  # noqa: E731
        rhs = s * b / np.linalg.norm(s * b)
        nrm = krylov.nrm2
        _, k1, _, _, h1 = krylov.cocg_inner(mv, rhs, 1e-12, 5000, 5000, None, nrm)
        _, k2, _, _, h2 = krylov.cocg_inner_qrec(mv, rhs, 1e-12, 5000, 5000, None, nrm)
        assert np.allclose(h1[:12], h2[:12], rtol=1e-8, atol=0)
        assert abs(k1 - k2) <= max(3, 0.1 * k1), (k1, k2)
        ref = np.linalg.solve(A.toarray(), b)
        y, st, outer = krylov.cocg_ir(mv, s * b, tol=1e-12, weights=w,
                                      inner=lambda s_, t_, im_, ml_, st_, nm_: krylov.cocg_inner_qrec(
                                          mv, s_, t_, im_, ml_, st_, nm_))
        assert st.converged and outer >= 1
        assert np.linalg.norm(s * y - ref) <= 1e-9 * np.linalg.norm(ref)


def test_residual_product_form_is_cg_on_spd():
    # real SPD (1D Laplacian): the recurrence form is CG, n steps in exact arithmetic
    n = 40
    A = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    b = np.random.default_rng(7).standard_normal(n) + 0j
    d, k, est, bd, _ = krylov.cocg_inner_qrec(lambda v: A @ v, b / np.linalg.norm(b), 1e-12, 200, 200, None,
                                             krylov.nrm2)
    assert not bd and est <= 1e-12 and k <= n + 2
    assert np.linalg.norm(A @ d - b / np.linalg.norm(b)) <= 1e-10
