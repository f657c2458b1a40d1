"""Pins of the oracle's boundary quads and wall term on every side of the box (CPU only).

The wall term of the Helmholtz operator (paper Sec. 3.2) is i k rho c B(beta) with B the
face mass of the admittance quads. These checks pin `oracle.mesh.boundary_quads` and
`oracle.fem.assemble_B` side by side, with unequal spacings h_x != h_y != h_z so that a
quad built on the wrong side, with the wrong spacings or in the wrong place of the
numbering fails:
  * uniform beta on one side gives exactly beta times the Kronecker product of the assembled
    1D mass matrices of the two in-plane axes and a unit corner matrix on the normal axis;
  * beta on a single quad lands on the four nodes the documented numbering names (sides
    x-, x+, y-, y+, z-, z+; inside a side u + n_u v, first remaining axis fastest), with the
    tensor face mass in vertex order (0,0), (1,0), (0,1), (1,1);
  * a duct along each axis, admittance on one end wall and a prescribed pressure on the
    other, is uniform across the duct and equals the exact 1D finite-element solution (a
    dense tridiagonal solve), and its continuum limit converges at O(h^2).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import helm_inputs as hi
from oracle import fem

SIDES = ("x-", "x+", "y-", "y+", "z-", "z+")


def mass_1d(n, h):
    """Assembled 1D linear-element mass matrix on n equal cells, written out entry by entry."""
    M = np.zeros((n + 1, n + 1))
    for i in range(n + 1):
        M[i, i] = ((i > 0) + (i < n)) * h / 3.0
        if i < n:
            M[i, i + 1] = M[i + 1, i] = h / 6.0
    return M


def corner(n, at_end):
    """(n+1)x(n+1) matrix with a single 1 at node 0 or node n."""
    E = np.zeros((n + 1, n + 1))
    E[n if at_end else 0, n if at_end else 0] = 1.0
    return E


def lattice(mesh):
    return (mesh.nx, mesh.ny, mesh.nz), (mesh.Lx / mesh.nx, mesh.Ly / mesh.ny, mesh.Lz / mesh.nz)


MESH = hi.Mesh(3, 4, 5, 0.9, 0.5, 1.3)  # h = 0.3, 0.125, 0.26


@pytest.mark.parametrize("side", range(6))
def test_uniform_side_admittance_is_a_kronecker_face_mass(side):
    N, H = lattice(MESH)
    off = MESH.side_offsets()
    beta = np.zeros(MESH.n_bfaces, dtype=np.complex128)
    bval = 0.3 - 0.7j
    beta[off[side]:off[side + 1]] = bval
    B = fem.assemble_B(MESH, beta).toarray()
    axis, at_end = side // 2, side % 2 == 1
    # per axis factor: the unit corner on the normal axis, the 1D mass on the two others
    f = [corner(N[a], at_end) if a == axis else mass_1d(N[a], H[a]) for a in range(3)]
    ref = bval * np.kron(f[2], np.kron(f[1], f[0]))  # node id i + (nx+1)(j + (ny+1) l)
    assert np.max(np.abs(B - ref)) <= 1e-15 * np.max(np.abs(ref))
    # the face's area, the sum of all entries
    area = np.prod([MESH.Lx, MESH.Ly, MESH.Lz]) / [MESH.Lx, MESH.Ly, MESH.Lz][axis]
    assert abs(B.sum() - bval * area) <= 1e-13 * area


def expected_quad(mesh, side, u, v):
    """The four node ids of quad (u, v) on `side` under the documented convention."""
    N = (mesh.nx, mesh.ny, mesh.nz)
    axis = side // 2
    rem = [a for a in range(3) if a != axis]  # first remaining axis is u (fastest)
    ids = []
    for dv in (0, 1):
        for du in (0, 1):
            ijk = [0, 0, 0]
            ijk[axis] = N[axis] if side % 2 else 0
            ijk[rem[0]] = u + du
            ijk[rem[1]] = v + dv
            ids.append(ijk[0] + (mesh.nx + 1) * (ijk[1] + (mesh.ny + 1) * ijk[2]))
    return ids


@pytest.mark.parametrize("side", range(6))
def test_single_quad_lands_where_the_numbering_says(side):
    N, H = lattice(MESH)
    off = MESH.side_offsets()
    axis = side // 2
    rem = [a for a in range(3) if a != axis]
    nu, nv = N[rem[0]], N[rem[1]]
    assert off[side + 1] - off[side] == nu * nv
    hu, hv = H[rem[0]], H[rem[1]]
    T = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    face = np.kron(T * hv, T * hu)  # vertex (a, b) numbered a + 2b, u fastest
    for (u, v) in [(0, 0), (nu - 1, 0), (0, nv - 1), (nu - 1, nv - 1), (nu // 2, nv // 2)]:
        beta = np.zeros(MESH.n_bfaces, dtype=np.complex128)
        beta[off[side] + u + nu * v] = 1.0
        B = fem.assemble_B(MESH, beta).tocoo()
        nodes = expected_quad(MESH, side, u, v)
        dense = np.zeros((MESH.n_nodes, MESH.n_nodes), dtype=np.complex128)
        dense[B.row, B.col] += B.data
        sub = dense[np.ix_(nodes, nodes)]
        assert np.max(np.abs(sub - face)) <= 1e-15
        mask = np.ones_like(dense, dtype=bool)
        mask[np.ix_(nodes, nodes)] = False
        assert not np.any(dense[mask]), (SIDES[side], u, v)


def admittance_1d(n, L, k, bhat, P, admittance_at_end):
    """Exact 1D FE solution of (K - k^2 M) p + i k bhat p_w e_w = 0 with the pressure P at the
    other end (w = 0, or w = n when `admittance_at_end`), by a dense solve."""
    h = L / n
    K = np.zeros((n + 1, n + 1))
    for i in range(n):
        K[i:i + 2, i:i + 2] += np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    A = (K - k * k * mass_1d(n, h)).astype(np.complex128)
    w, d = (n, 0) if admittance_at_end else (0, n)
    A[w, w] += 1j * k * bhat
    free = [i for i in range(n + 1) if i != d]
    p = np.empty(n + 1, dtype=np.complex128)
    p[free] = np.linalg.solve(A[np.ix_(free, free)], -A[free, d] * P)
    p[d] = P
    return p


def duct(side, n_along, L_along, beta, P):
    """Duct along the side's normal axis: admittance on `side`, pressure P on the opposite wall,
    the other four walls rigid; transverse lattice 2 x 3 with unequal spacings."""
    axis = side // 2
    N = [2, 3, 2]
    Ls = [0.35, 0.6, 0.45]
    N[axis] = n_along
    Ls[axis] = L_along
    mesh = hi.Mesh(N[0], N[1], N[2], *Ls)
    off = mesh.side_offsets()
    b = np.zeros(mesh.n_bfaces, dtype=np.complex128)
    b[off[side]:off[side + 1]] = beta
    at = 0 if side % 2 else N[axis]  # the opposite wall
    ids = np.arange(mesh.n_nodes)
    ijk = (ids % (N[0] + 1), (ids // (N[0] + 1)) % (N[1] + 1), ids // ((N[0] + 1) * (N[1] + 1)))
    dnodes = ids[ijk[axis] == at].astype(np.int32)
    return hi.Problem(mesh, b, dnodes, np.full(len(dnodes), P, dtype=np.complex128)), ijk


def profile(p, ijk, axis, n):
    """Pressure along the axis, after checking that it is uniform across the duct."""
    out = np.empty(n + 1, dtype=np.complex128)
    for i in range(n + 1):
        sel = p[ijk[axis] == i]
        assert np.max(np.abs(sel - sel[0])) <= 1e-11 * max(1.0, np.max(np.abs(p)))
        out[i] = sel[0]
    return out


@pytest.mark.parametrize("side", range(6))
def test_admittance_duct_on_every_side_is_the_exact_1d_solution(side):
    P, f, L, beta = 0.7 + 0.2j, 110.0, 1.1, 0.003 + 0.002j
    k = 2 * np.pi * f / hi.C_SOUND
    bhat = hi.RHO_AIR * hi.C_SOUND * beta
    n = 9
    prob, ijk = duct(side, n, L, beta, P)
    A, b = fem.system(prob, f)
    p = spl.spsolve(A.tocsc(), b)
    axis = side // 2
    got = profile(p, ijk, axis, n)
    ref = admittance_1d(n, L, k, bhat, P, admittance_at_end=side % 2 == 1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), SIDES[side]


@pytest.mark.parametrize("side", (0, 3, 5))
def test_admittance_duct_continuum_limit_at_h2(side):
    # continuum: p'' + k^2 p = 0, admittance wall at distance s = 0 with p'(0) = i k bhat p(0)
    # (outward normal pointing out of the duct), pressure P at s = L:
    # p(s) = P (cos ks + i bhat sin ks) / (cos kL + i bhat sin kL)
    P, f, L, beta = 1.0 - 0.5j, 95.0, 1.0, 0.002 + 0.001j
    k = 2 * np.pi * f / hi.C_SOUND
    bhat = hi.RHO_AIR * hi.C_SOUND * beta
    errs = []
    for n in (10, 20, 40):
        prob, ijk = duct(side, n, L, beta, P)
        A, b = fem.system(prob, f)
        got = profile(spl.spsolve(A.tocsc(), b), ijk, side // 2, n)
        x = np.linspace(0.0, L, n + 1)
        s = L - x if side % 2 else x  # distance from the admittance wall
        cont = P * (np.cos(k * s) + 1j * bhat * np.sin(k * s)) / (np.cos(k * L) + 1j * bhat * np.sin(k * L))
        errs.append(np.linalg.norm(got - cont) / np.linalg.norm(cont))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3
