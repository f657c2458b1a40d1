"""Pins of the oracle's Schwarz preconditioners with Robin (absorbing) interface terms: the
interface face mass against its closed Kronecker form, a single block is the exact inverse, and
GMRES with the preconditioner reaches the direct solution."""
import numpy as np

import helm_inputs as hi
from oracle import fem, krylov, ras
def test_interface_mass_is_the_kronecker_face_mass():
    # closed form: on a face plane the Q1 face mass is M1(h_u) (x) M1(h_v), M1(h) the 1D linear
    # mass (h/6)[[2,1],[1,2]] assembled over the face's extent; only faces inside the lattice count
    mesh = hi.Mesh(6, 5, 4, 1.2, 0.8, 0.9)
    dims = (7, 6, 5)
    # x- face at i=2, y+ face at j=3 and z- face at l=1 lie inside; x+, y-, z+ are on the walls
    ext = ((2, 7), (0, 4), (1, 5))
    Mg = ras.interface_mass(mesh, ext).toarray()
    h = (1.2 / 6, 0.8 / 5, 0.9 / 4)

    def m1(lo, hi_, hh):
        n = hi_ - lo
        M = np.zeros((n, n))
        for e in range(n - 1):
            M[e:e + 2, e:e + 2] += hh / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
        return M

    ref = np.zeros_like(Mg)
    for a, plane in ((0, 2), (1, 3), (2, 1)):
        u, v = [b for b in range(3) if b != a]
        Mu, Mv = m1(*ext[u], h[u]), m1(*ext[v], h[v])
        for iu in range(ext[u][1] - ext[u][0]):
            for iv in range(ext[v][1] - ext[v][0]):
                for ju in range(ext[u][1] - ext[u][0]):
                    for jv in range(ext[v][1] - ext[v][0]):
                        p, q = [0, 0, 0], [0, 0, 0]
                        p[a] = q[a] = plane
                        p[u], p[v] = ext[u][0] + iu, ext[v][0] + iv
                        q[u], q[v] = ext[u][0] + ju, ext[v][0] + jv
                        r = p[0] + dims[0] * (p[1] + dims[1] * p[2])
                        c = q[0] + dims[0] * (q[1] + dims[1] * q[2])
                        ref[r, c] += Mu[iu, ju] * Mv[iv, jv]
    assert np.abs(Mg - ref).max() <= 1e-15
    # total = the interface area: 0.48 x 0.675 + 0.8 x 0.675 + 0.8 x 0.48
    assert abs(Mg.sum() - (0.48 * 0.675 + 0.8 * 0.675 + 0.8 * 0.48)) <= 1e-14


def test_robin_schwarz_single_block_and_convergence():
    prob = hi.small_box_problem(12, 8, 6)
    f = 180.0
    A, b = fem.system(prob, f)
    k = 2 * np.pi * f / prob.c
    ref = np.linalg.solve(A.toarray(), b)
    # one block: no artificial interface, the Robin term vanishes and the preconditioner is A^-1
    P1 = ras.RAS(A, prob.mesh, (1, 1, 1), 2, robin=1j * k, dir_nodes=prob.dir_nodes)
    x, st = krylov.gmres(lambda v: A @ v, b, 30, 1e-12, precond=P1)
    assert st.iterations == 1 and np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    # several blocks: GMRES with the Robin-interface preconditioner reaches the direct solution
    P = ras.RAS(A, prob.mesh, (3, 2, 2), 1, robin=1j * k, dir_nodes=prob.dir_nodes)
    x, st = krylov.gmres(lambda v: A @ v, b, 30, 1e-12, maxit=3000, precond=P)
    assert st.converged and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_two_sided_face_masses_split_the_interface_mass():
    # low faces + high faces = every interface face; "scaled" divides each face by the spacing
    # normal to it; a one-layer box counts its single plane once, as a low face
    mesh = hi.Mesh(6, 5, 4, 1.2, 0.8, 0.9)
    h = (1.2 / 6, 0.8 / 5, 0.9 / 4)
    ext = ((2, 7), (0, 4), (1, 5))
    both = ras.interface_mass(mesh, ext).toarray()
    lo = ras.interface_mass(mesh, ext, "lo").toarray()
    hi_ = ras.interface_mass(mesh, ext, "hi").toarray()
    assert np.abs(both - lo - hi_).max() <= 1e-17
    # the low faces here are x at i=2 and z at l=1, the high face y at j=3
    assert abs(lo.sum() - (0.48 * 0.675 + 0.8 * 0.48)) <= 1e-14
    assert abs(hi_.sum() - 0.8 * 0.675) <= 1e-14
    slo = ras.interface_mass(mesh, ext, "lo", scaled=True).toarray()
    assert abs(slo.sum() - (0.48 * 0.675 / h[0] + 0.8 * 0.48 / h[2])) <= 1e-12
    thin = ((3, 4), (0, 6), (0, 5))  # one x-layer inside the lattice
    assert abs(ras.interface_mass(mesh, thin, "lo").toarray().sum() - 0.8 * 0.9) <= 1e-14
    assert ras.interface_mass(mesh, thin, "hi").nnz == 0
    assert np.abs(ras.interface_mass(mesh, thin).toarray() - ras.interface_mass(mesh, thin, "lo").toarray()).max() == 0


def test_two_sided_robin_schwarz():
    prob = hi.small_box_problem(10, 8, 6)  # isotropic lattice: h = 0.1 on every axis
    m = prob.mesh
    h = m.Lx / m.nx
    assert abs(m.Ly / m.ny - h) < 1e-15 and abs(m.Lz / m.nz - h) < 1e-15
    f = 180.0
    A, b = fem.system(prob, f)
    ref = np.linalg.solve(A.toarray(), b)
    r = np.random.default_rng(5).standard_normal(A.shape[0]) + 0j
    c = np.exp(0.75j * np.pi)
    # equal coefficients on both sides: the one-sided preconditioner with robin = c / h
    P2 = ras.RAS(A, m, (3, 2, 2), 1, robin=(c, c), dir_nodes=prob.dir_nodes)
    P1 = ras.RAS(A, m, (3, 2, 2), 1, robin=c / h, dir_nodes=prob.dir_nodes)
    assert np.linalg.norm(P2(r) - P1(r)) <= 1e-12 * np.linalg.norm(P1(r))
    # different sides: a different preconditioner, still exact for one block, still converging
    Pc = ras.RAS(A, m, (3, 2, 2), 1, robin=(c, np.conj(c)), dir_nodes=prob.dir_nodes)
    assert np.linalg.norm(Pc(r) - P1(r)) > 1e-6 * np.linalg.norm(P1(r))
    Pone = ras.RAS(A, m, (1, 1, 1), 2, robin=(c, np.conj(c)), dir_nodes=prob.dir_nodes)
    x, st = krylov.gmres(lambda v: A @ v, b, 30, 1e-12, precond=Pone)
    assert st.iterations == 1 and np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    x, st = krylov.gmres(lambda v: A @ v, b, 30, 1e-12, maxit=3000, precond=Pc)
    assert st.converged and np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
