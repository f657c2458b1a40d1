"""Pins of the oracle's double-word arithmetic (oracle/dwfloat.py), CPU only.

The error-free transformations are checked exact against rational arithmetic; the double-word
multiply-add accumulation, the stencil product and the complex axpy against their exact values
within the error bound of the format (about 2^-44 of the sum of magnitudes for a 27-term Dot2
accumulation of double-word operands, against 2^-24 for plain float32); the inner COCG in this
arithmetic, run through the refinement, against dense LU.
"""
from fractions import Fraction

import numpy as np
import pytest

import helm_inputs as hi
from oracle import dwfloat as dw
from oracle import fem, krylov

f32 = np.float32


def rand32(rng, n, spread=8):
    return (rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread, n)).astype(f32)


def test_two_sum_and_two_prod_are_error_free():
    rng = np.random.default_rng(0)
    a, b = rand32(rng, 2000), rand32(rng, 2000)
    s, e = dw.two_sum(a, b)
    for i in range(0, 2000, 7):
        assert Fraction(float(s[i])) + Fraction(float(e[i])) == Fraction(float(a[i])) + Fraction(float(b[i]))
    big, small = np.where(np.abs(a) >= np.abs(b), a, b), np.where(np.abs(a) >= np.abs(b), b, a)
    s, e = dw.fast_two_sum(big, small)
    for i in range(0, 2000, 7):
        assert Fraction(float(s[i])) + Fraction(float(e[i])) == Fraction(float(big[i])) + Fraction(float(small[i]))
    p = a * b
    e = dw.fma(a, b, -p)
    for i in range(0, 2000, 7):
        assert Fraction(float(p[i])) + Fraction(float(e[i])) == Fraction(float(a[i])) * Fraction(float(b[i]))


def test_split_carries_about_48_bits():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(5000) * 10.0 ** rng.integers(-5, 5, 5000)
    hi, lo = dw.split(v)
    assert np.array_equal(hi, v.astype(f32))
    assert np.max(np.abs(dw.join(hi, lo) - v) / np.abs(v)) <= 2.0 ** -47


def test_dot2_accumulation_of_27_double_word_products():
    # 27-term dot products with cancellation (stencil-like: a positive centre, negative ring)
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(200):
        a = rng.standard_normal(27)
        a[13] = -np.sum(a) + rng.standard_normal() * 1e-3
        x = rng.standard_normal(27)
        ah, al = dw.split(a)
        xh, xl = dw.split(x)
        acc = dw.Acc.zeros(1)
        for k in range(27):
            acc.mac(ah[k:k + 1], al[k:k + 1], xh[k:k + 1], xl[k:k + 1])
        h, l = acc.get()
        exact = sum(Fraction(float(dw.join(ah[k:k + 1], al[k:k + 1])[0])) *
                    Fraction(float(dw.join(xh[k:k + 1], xl[k:k + 1])[0])) for k in range(27))
        mag = sum(abs(float(a[k] * x[k])) for k in range(27))
        err = abs(float(Fraction(float(h[0])) + Fraction(float(l[0])) - exact)) / mag
        worst = max(worst, err)
    assert worst <= 2.0 ** -44, worst


def test_complex_axpy_within_double_word_precision():
    rng = np.random.default_rng(3)
    n = 4000
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a = 0.37 - 1.9j
    Y, X = dw.CW.from_complex(y), dw.CW.from_complex(x)
    got = dw.axpy(Y, a, X).to_complex()
    exact = Y.to_complex() + complex(*map(float, (dw.join(*dw.split(np.array([a.real])))[0],
                                                  dw.join(*dw.split(np.array([a.imag])))[0]))) * X.to_complex()
    scale = np.abs(Y.to_complex()) + abs(a) * np.abs(X.to_complex())
    assert np.max(np.abs(got - exact) / scale) <= 2.0 ** -45


@pytest.mark.parametrize("dims,f", [((6, 4, 3), 230.0), ((9, 5, 4), 120.0)])
def test_stencil_product_matches_the_fp64_product(dims, f):
    prob = hi.cabin_problem(*dims)
    A, _ = fem.system(prob, f)
    Ah, _, _ = krylov.sym_jacobi(A)
    m = prob.mesh
    slots = dw.slots_from_csr(Ah, m.nx, m.ny)
    # the slot arrays hold exactly the matrix (each entry once, in the slot of its offset)
    assert np.count_nonzero(slots) == Ah.count_nonzero()
    M = dw.StencilMatrix(slots, m.nx, m.ny)
    assert M.cplx.any() and not M.cplx.all()  # admittance rows take the second pass
    rng = np.random.default_rng(4)
    x = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    X = dw.CW.from_complex(x)
    q = M.matvec(X).to_complex()
    xe = X.to_complex()
    ref = Ah @ xe
    bound = np.abs(Ah) @ np.abs(xe)
    assert np.max(np.abs(q - ref) / bound) <= 2.0 ** -43


@pytest.mark.parametrize("dims,f", [((6, 4, 3), 230.0), ((10, 8, 6), 150.0)])
def test_double_word_inner_solve_through_refinement_matches_dense_lu(dims, f):
    prob = hi.small_box_problem(*dims)
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    Ah, s, w = krylov.sym_jacobi(A)
    m = prob.mesh
    M = dw.StencilMatrix(dw.slots_from_csr(Ah, m.nx, m.ny), m.nx, m.ny)
    mv = lambda v: Ah @ v
    y, st, outer = krylov.cocg_ir(mv, s * b, tol=1e-12, weights=w, inner=dw.make_inner(M))
    assert st.converged and outer >= 1
    assert np.linalg.norm(s * y - ref) <= 1e-9 * np.linalg.norm(ref)
    # at the sweep's target the double-word inner solve takes about the FP64 one's steps
    _, st_dw, o1 = krylov.cocg_ir(mv, s * b, tol=1e-10, weights=w, inner=dw.make_inner(M))
    _, st_64, o2 = krylov.cocg_ir(mv, s * b, tol=1e-10, weights=w)
    assert o1 == o2 == 1
    assert abs(st_dw.iterations - st_64.iterations) <= max(2, 0.05 * st_64.iterations)


def test_double_word_inner_solve_in_the_residual_product_form():
    # form="qrec" follows krylov.cocg_inner_qrec in double-word arithmetic: its first residual
    # estimates agree with the plain double-word inner solve's to the format's rounding, and the
    # refinement around it reaches the dense-LU solution
    prob = hi.small_box_problem(10, 8, 6)
    A, b = fem.system(prob, 150.0)
    ref = np.linalg.solve(A.toarray(), b)
    Ah, s, w = krylov.sym_jacobi(A)
    m = prob.mesh
    M = dw.StencilMatrix(dw.slots_from_csr(Ah, m.nx, m.ny), m.nx, m.ny)
    rhs = s * b / np.linalg.norm(s * b)
    _, k1, _, _, h1 = dw.make_inner(M)(rhs, 1e-12, 5000, 5000, None, krylov.nrm2)
    _, k2, _, _, h2 = dw.make_inner(M, form="qrec")(rhs, 1e-12, 5000, 5000, None, krylov.nrm2)
    assert np.allclose(h1[:12], h2[:12], rtol=1e-8, atol=0)
    assert abs(k1 - k2) <= max(3, 0.1 * k1), (k1, k2)
    y, st, outer = krylov.cocg_ir(lambda v: Ah @ v, s * b, tol=1e-12, weights=w, inner=dw.make_inner(M, form="qrec"))
    assert st.converged and outer >= 1
    assert np.linalg.norm(s * y - ref) <= 1e-9 * np.linalg.norm(ref)
