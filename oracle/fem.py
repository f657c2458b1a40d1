"""Q1 finite-element Helmholtz operator on the box lattice (oracle; test infrastructure).

Paper Sec. 3.2: the wave equation in the compartment becomes, after the Fourier
transform in time, the Helmholtz equation -w^2 psi - c^2 lap(psi) = 0 (Helmholtz eq.),
solved by finite elements with the sun-roof pressure as Dirichlet data. Discretised with
trilinear (Q1) bricks this is (K - k^2 M) p = 0, k = w / c, plus a wall term
i k rho c B(beta) for admittance faces (sign reading: dissipative for Re beta > 0 under
the e^{+i w t} convention).

Element integrals use 2x2x2 Gauss-Legendre quadrature on the reference cube (exact for
Q1 on bricks); face integrals use 2x2 Gauss. Assembly is a plain scatter-add of element
matrices (duplicates summed by scipy).

Pinned (tests/test_oracle_fem.py): element matrices equal their tensor closed forms;
assembled K, M equal the Kronecker products of the assembled 1D matrices; A == A^T;
discrete rigid-box eigenpairs are exact tensor cosines; discrete duct and admittance-duct
solutions are exact 1D recurrences; continuum duct / eigenfrequencies converge at O(h^2).
"""
import numpy as np
import scipy.sparse as sp

from . import mesh as _mesh

_G = np.array([-1.0, 1.0]) / np.sqrt(3.0)  # 2-point Gauss-Legendre nodes on [-1,1], weights 1


def _shape_1d(t):
    """Linear Lagrange shapes on [-1,1] at t: (N0, N1), and their t-derivatives."""
    return np.array([(1 - t) / 2, (1 + t) / 2]), np.array([-0.5, 0.5])


def brick_matrices(hx, hy, hz):
    """8x8 stiffness K_e = int grad Ni . grad Nj and mass M_e = int Ni Nj on an hx*hy*hz brick."""
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    jac = np.array([hx / 2, hy / 2, hz / 2])
    detJ = jac.prod()
    for tx in _G:
        for ty in _G:
            for tz in _G:
                Nx, dNx = _shape_1d(tx)
                Ny, dNy = _shape_1d(ty)
                Nz, dNz = _shape_1d(tz)
                N = np.zeros(8)
                G = np.zeros((8, 3))
                for c in (0, 1):
                    for b in (0, 1):
                        for a in (0, 1):
                            q = a + 2 * b + 4 * c
                            N[q] = Nx[a] * Ny[b] * Nz[c]
                            # physical gradient = reference gradient / (h/2)
                            G[q] = [dNx[a] * Ny[b] * Nz[c] / jac[0],
                                    Nx[a] * dNy[b] * Nz[c] / jac[1],
                                    Nx[a] * Ny[b] * dNz[c] / jac[2]]
                Ke += G @ G.T * detJ
                Me += np.outer(N, N) * detJ
    return Ke, Me


def quad_mass(hu, hv):
    """4x4 face mass int Ni Nj dS on an hu*hv quad, vertex (a,b) numbered a + 2b."""
    Bf = np.zeros((4, 4))
    detJ = hu * hv / 4
    for tu in _G:
        for tv in _G:
            Nu, _ = _shape_1d(tu)
            Nv, _ = _shape_1d(tv)
            N = np.array([Nu[a] * Nv[b] for b in (0, 1) for a in (0, 1)])
            Bf += np.outer(N, N) * detJ
    return Bf


def assemble_KM(mesh):
    """Global stiffness K and mass M (real CSR) by scatter-add over all bricks."""
    Ke, Me = brick_matrices(mesh.Lx / mesh.nx, mesh.Ly / mesh.ny, mesh.Lz / mesh.nz)
    conn = _mesh.bricks(mesh)
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    n = mesh.n_nodes
    K = sp.coo_matrix((np.tile(Ke.ravel(), len(conn)), (rows, cols)), shape=(n, n)).tocsr()
    M = sp.coo_matrix((np.tile(Me.ravel(), len(conn)), (rows, cols)), shape=(n, n)).tocsr()
    return K, M


def assemble_B(mesh, beta):
    """Admittance matrix B(beta) = sum_f beta_f int_f Ni Nj dS (complex CSR), beta per boundary quad."""
    quads = _mesh.boundary_quads(mesh)
    rows, cols, vals = [], [], []
    for f, (nodes, (hu, hv)) in enumerate(quads):
        if beta[f] == 0:
            continue
        Bf = quad_mass(hu, hv)
        for a in range(4):
            for b in range(4):
                rows.append(nodes[a])
                cols.append(nodes[b])
                vals.append(beta[f] * Bf[a, b])
    n = mesh.n_nodes
    return sp.coo_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(n, n)).tocsr()


def wavenumber(freq, c):
    return 2.0 * np.pi * freq / c


def helmholtz_matrix(prob, freq, KM=None):
    """A = K - k^2 M + i k rho c B(beta) before Dirichlet elimination (complex CSR)."""
    K, M = KM if KM is not None else assemble_KM(prob.mesh)
    B = assemble_B(prob.mesh, prob.beta)
    k = wavenumber(freq, prob.c)
    return (K - k * k * M + 1j * k * prob.rho * prob.c * B).tocsr().astype(np.complex128)


def eliminate_dirichlet(A, dir_nodes, p_dir):
    """Symmetric elimination of prescribed nodes D (paper Sec. 3.2: sun-roof Dirichlet data).

    Returns (A_red, b): A_red has identity rows/columns on D and A_FF elsewhere;
    b_F = -A_FD p_D, b_D = p_D. A_red stays complex symmetric.
    """
    n = A.shape[0]
    isD = np.zeros(n, dtype=bool)
    isD[np.asarray(dir_nodes)] = True
    xD = np.zeros(n, dtype=np.complex128)
    xD[dir_nodes] = p_dir
    b = -(A @ xD)
    b[isD] = p_dir
    keep = sp.diags((~isD).astype(np.float64))
    A_red = (keep @ A @ keep + sp.diags(isD.astype(np.float64))).tocsr()
    return A_red, b


def system(prob, freq, KM=None):
    """The linear system (A_red, b) one frequency of the frequency-response sweep solves."""
    A = helmholtz_matrix(prob, freq, KM)
    return eliminate_dirichlet(A, prob.dir_nodes, prob.p_dir)
