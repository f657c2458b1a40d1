"""Pins of the oracle's FE operator against what the mathematics fixes (CPU only).

Each check is a closed form or an invariant independent of the oracle's own code path
(quadrature + scatter-add): tensor-product closed forms, Kronecker structure of the
assembled box-lattice matrices, exact discrete eigenpairs and 1D recurrences, and the
O(h^2) convergence to the continuum duct / rigid-box solutions.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import helm_inputs as hi
from oracle import fem


def k1(h):
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def m1(h):
    return np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0


def test_brick_matrices_equal_tensor_closed_form():
    hx, hy, hz = 0.3, 0.7, 1.1
    Ke, Me = fem.brick_matrices(hx, hy, hz)
    # local vertex a + 2b + 4c: x fastest -> kron(z, kron(y, x))
    K_ref = (np.kron(m1(hz), np.kron(m1(hy), k1(hx))) + np.kron(m1(hz), np.kron(k1(hy), m1(hx)))
             + np.kron(k1(hz), np.kron(m1(hy), m1(hx))))
    M_ref = np.kron(m1(hz), np.kron(m1(hy), m1(hx)))
    assert np.max(np.abs(Ke - K_ref)) <= 1e-15 * np.max(np.abs(K_ref)) * 10
    assert np.max(np.abs(Me - M_ref)) <= 1e-15 * np.max(np.abs(M_ref)) * 10
    # row sums of K vanish (constants are in the kernel); M sums to the brick volume
    assert np.max(np.abs(Ke.sum(1))) < 1e-14
    assert abs(Me.sum() - hx * hy * hz) < 1e-15


def test_quad_mass_closed_form():
    hu, hv = 0.25, 0.6
    B = fem.quad_mass(hu, hv)
    assert np.max(np.abs(B - np.kron(m1(hv), m1(hu)))) < 1e-16
    assert abs(B.sum() - hu * hv) < 1e-15


def assembled_1d(n, h):
    """Assembled 1D linear-element stiffness and mass on n equal cells (written out)."""
    K = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    for i in range(n + 1):
        cells = (i > 0) + (i < n)
        K[i, i] = cells / h
        M[i, i] = cells * h / 3.0
        if i < n:
            K[i, i + 1] = K[i + 1, i] = -1.0 / h
            M[i, i + 1] = M[i + 1, i] = h / 6.0
    return K, M


def test_assembled_matrices_are_kronecker_products():
    mesh = hi.Mesh(4, 3, 2, 1.0, 0.8, 0.6)
    K, M = fem.assemble_KM(mesh)
    Kx, Mx = assembled_1d(4, 0.25)
    Ky, My = assembled_1d(3, 0.8 / 3)
    Kz, Mz = assembled_1d(2, 0.3)
    # node id = i + (nx+1)(j + (ny+1) l): x fastest
    K_ref = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    M_ref = np.kron(Mz, np.kron(My, Mx))
    assert np.max(np.abs(K.toarray() - K_ref)) < 1e-14
    assert np.max(np.abs(M.toarray() - M_ref)) < 1e-16
    # full 27-point pattern (interior rows 27 entries)
    assert K.nnz == mesh.nnz27


def test_helmholtz_matrix_symmetric_exactly():
    prob = hi.small_box_problem()
    A = fem.helmholtz_matrix(prob, 100.0)
    assert abs(A - A.T).max() == 0.0
    A_red, b = fem.eliminate_dirichlet(A, prob.dir_nodes, prob.p_dir)
    assert abs(A_red - A_red.T).max() == 0.0
    assert A.shape == (4641, 4641)


def lam_h(l, n, h):
    th = np.pi * l / n
    return (6.0 / h ** 2) * (1 - np.cos(th)) / (2 + np.cos(th))


def test_rigid_box_discrete_eigenpairs_exact():
    mesh = hi.Mesh(6, 5, 4, 1.0, 0.8, 0.6)
    K, M = fem.assemble_KM(mesh)
    hx, hy, hz = 1.0 / 6, 0.8 / 5, 0.6 / 4
    i = np.arange(7)[None, None, :]
    j = np.arange(6)[None, :, None]
    l = np.arange(5)[:, None, None]
    for (a, b, c) in [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (2, 3, 1), (5, 4, 3)]:
        v = (np.cos(np.pi * a * i / 6) * np.cos(np.pi * b * j / 5) * np.cos(np.pi * c * l / 4)).ravel()
        lam = lam_h(a, 6, hx) + lam_h(b, 5, hy) + lam_h(c, 4, hz)
        res = K @ v - lam * (M @ v)
        assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(K @ v) + 1e-13


def test_rigid_box_spectrum_is_exactly_the_tensor_cosines():
    # dense generalised eigenproblem (library routine) on a small lattice: every eigenvalue is
    # one of the tensor-cosine values, none missing
    mesh = hi.Mesh(5, 4, 3, 1.0, 0.8, 0.6)
    K, M = fem.assemble_KM(mesh)
    ev = np.sort(sla.eigh(K.toarray(), M.toarray(), eigvals_only=True))
    ref = np.sort([lam_h(a, 5, 0.2) + lam_h(b, 4, 0.2) + lam_h(c, 3, 0.2)
                   for a in range(6) for b in range(5) for c in range(4)])
    assert np.max(np.abs(ev - ref)) <= 1e-9 * ref.max()


def test_rigid_box_eigenfrequencies_converge_at_h2():
    # (1,0,0) mode of the 1.0 x 0.8 x 0.6 box: continuum f = c/2 * 1/Lx = 170 Hz
    errs = []
    for nx in (10, 20, 40):
        f_h = hi.C_SOUND / (2 * np.pi) * np.sqrt(lam_h(1, nx, 1.0 / nx))
        errs.append(abs(f_h - 170.0))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2
    # on the 20-cell axis of the 20x16x12 lattice the (1,0,0) mode sits at 170.17 Hz (continuum 170.0 Hz)
    f20 = hi.C_SOUND / (2 * np.pi) * np.sqrt(lam_h(1, 20, 0.05))
    assert abs(f20 - 170.17) < 0.01


def duct_problem(nx, ny, nz, Lz, P, beta_floor=0.0):
    mesh = hi.Mesh(nx, ny, nz, 0.5, 0.4, Lz)
    top = np.array([i + (nx + 1) * (j + (ny + 1) * nz) for j in range(ny + 1) for i in range(nx + 1)],
                   dtype=np.int32)
    beta = np.zeros(mesh.n_bfaces, dtype=np.complex128)
    off = mesh.side_offsets()
    beta[off[4]:off[5]] = beta_floor
    return hi.Problem(mesh, beta, np.sort(top), np.full(len(top), P, dtype=np.complex128))


def z_profile(p, mesh):
    """Pressure along the lattice z-line at i=j=0, and check it is uniform in x, y."""
    P3 = p.reshape(mesh.nz + 1, mesh.ny + 1, mesh.nx + 1)
    assert np.max(np.abs(P3 - P3[:, :1, :1])) <= 1e-11 * np.max(np.abs(P3))
    return P3[:, 0, 0]


def test_discrete_duct_exact_recurrence():
    nz, Lz, P, f = 10, 1.0, 1.3 - 0.4j, 130.0
    prob = duct_problem(3, 2, nz, Lz, P)
    A_red, b = fem.system(prob, f)
    p = spl.spsolve(A_red.tocsc(), b)
    k, h = 2 * np.pi * f / hi.C_SOUND, Lz / nz
    th = np.arccos((6 - 2 * k * k * h * h) / (6 + k * k * h * h))
    ref = P * np.cos(th * np.arange(nz + 1)) / np.cos(th * nz)
    pz = z_profile(p, prob.mesh)
    assert np.max(np.abs(pz - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_continuum_duct_converges_at_h2():
    P, f, Lz = 1.0, 130.0, 1.0
    k = 2 * np.pi * f / hi.C_SOUND
    errs = []
    for nz in (10, 20, 40):
        prob = duct_problem(1, 1, nz, Lz, P)
        A_red, b = fem.system(prob, f)
        pz = z_profile(spl.spsolve(A_red.tocsc(), b), prob.mesh)
        z = np.linspace(0, Lz, nz + 1)
        ref = P * np.cos(k * z) / np.cos(k * Lz)
        errs.append(np.linalg.norm(pz - ref) / np.linalg.norm(ref))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3


def admittance_1d(nz, Lz, k, bhat, P):
    """1D FE system (K - k^2 M) p + i k bhat p_0 e_0 = 0, p_nz = P, solved densely."""
    K, M = assembled_1d(nz, Lz / nz)
    A = (K - k * k * M).astype(np.complex128)
    A[0, 0] += 1j * k * bhat
    rhs = -A[:nz, nz] * P
    p = np.empty(nz + 1, dtype=np.complex128)
    p[:nz] = np.linalg.solve(A[:nz, :nz], rhs)
    p[nz] = P
    return p


def test_admittance_duct_discrete_exact_and_continuum_h2():
    P, f, Lz, beta = 0.7 + 0.2j, 90.0, 1.0, 0.002 + 0.001j
    k = 2 * np.pi * f / hi.C_SOUND
    bhat = hi.RHO_AIR * hi.C_SOUND * beta
    errs = []
    for nz in (10, 20, 40):
        prob = duct_problem(2, 1, nz, Lz, P, beta_floor=beta)
        A_red, b = fem.system(prob, f)
        pz = z_profile(spl.spsolve(A_red.tocsc(), b), prob.mesh)
        ref1d = admittance_1d(nz, Lz, k, bhat, P)
        assert np.max(np.abs(pz - ref1d)) <= 1e-12 * np.max(np.abs(ref1d))
        z = np.linspace(0, Lz, nz + 1)
        cont = P * (np.cos(k * z) + 1j * bhat * np.sin(k * z)) / (np.cos(k * Lz) + 1j * bhat * np.sin(k * Lz))
        errs.append(np.linalg.norm(pz - cont) / np.linalg.norm(cont))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3


def test_elimination_equals_constrained_solve():
    prob = hi.small_box_problem(8, 6, 5)
    A = fem.helmholtz_matrix(prob, 180.0)
    A_red, b = fem.eliminate_dirichlet(A, prob.dir_nodes, prob.p_dir)
    p = spl.spsolve(A_red.tocsc(), b)
    D = prob.dir_nodes
    F = np.setdiff1d(np.arange(A.shape[0]), D)
    pF = spl.spsolve(A[F][:, F].tocsc(), -(A[F][:, D] @ prob.p_dir))
    assert np.max(np.abs(p[D] - prob.p_dir)) == 0.0
    assert np.max(np.abs(p[F] - pF)) <= 1e-12 * np.max(np.abs(pF))


def test_sign_of_admittance_is_dissipative():
    # with Re beta > 0 and e^{+i w t}, the wall absorbs: time-averaged power into the domain
    # through the Dirichlet patch is positive, i.e. Im(p_D^H (A p)_D) has the sign of -Re(...)
    # Simplest invariant: the energy balance Im(p^H A p) = k rho c Re(beta) ||p||_B^2 > 0 for a
    # uniform floor beta.
    prob = hi.small_box_problem(6, 5, 4)
    A = fem.helmholtz_matrix(prob, 100.0)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    val = np.vdot(p, A @ p)
    assert val.imag > 0


def test_golden_box_modes_from_the_oracle_assembly():
    """tests/golden/box_modes.json holds closed-form mode frequencies of the rigid test box and
    cabin (written by tests/golden/make_box_modes.py from the formulas alone). The oracle's
    assembled K, M reproduce the discrete ones (generalised eigenproblem) to 1e-9, and the
    discrete values lie within 1% of the continuum ones at these lattices."""
    import importlib.util
    import json
    import os

    import scipy.sparse.linalg as spl

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    stored = json.load(open(os.path.join(here, "box_modes.json")))
    spec = importlib.util.spec_from_file_location("make_box_modes", os.path.join(here, "make_box_modes.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    for name, (L, N) in gen.BOXES.items():
        assert gen.modes(L, N) == stored["boxes"][name]["modes"]  # the fixture is the formula's output
        mesh = hi.Mesh(N[0], N[1], N[2], *L)
        K, M = fem.assemble_KM(mesh)
        modes = stored["boxes"][name]["modes"]
        fd = np.array([m["f_discrete"] for m in modes])
        # shift-invert around the stored band; the rigid box has the constant mode at 0
        sigma = (2 * np.pi * fd[0] * 0.5 / stored["c"]) ** 2
        vals = spl.eigsh(K.tocsc(), k=len(fd) + 1, M=M.tocsc(), sigma=sigma, which="LM", return_eigenvectors=False)
        f_oracle = np.sort(stored["c"] * np.sqrt(np.clip(vals, 0, None)) / (2 * np.pi))
        f_oracle = f_oracle[f_oracle > 1.0][:len(fd)]
        assert np.allclose(f_oracle, fd, rtol=1e-9, atol=0), (name, f_oracle, fd)
        fc = np.array([m["f_continuum"] for m in modes])
        assert np.all(np.abs(fd - fc) <= 0.01 * fc)
