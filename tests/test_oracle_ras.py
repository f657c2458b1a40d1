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
