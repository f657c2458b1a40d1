"""Box lattice of Q1 bricks (oracle; test infrastructure).

Follows the paper's Sec. 3.2 FE discretisation of the compartment, restated on a
structured box lattice: node id = i + (nx+1)(j + (ny+1) l); brick (i,j,l) has local
vertices (a,b,c) in {0,1}^3 numbered a + 2b + 4c; boundary quads are numbered side by
side x-, x+, y-, y+, z-, z+ and, inside a side, by u + nu*v over the two remaining axes
(first remaining axis fastest). Pinned by tests/test_oracle_fem.py (assembled matrices
equal the Kronecker closed form, which depends on this numbering) and, quad by quad and side
by side, by tests/test_oracle_boundary.py (face mass of every side equals its Kronecker
closed form; single quads land on the nodes the numbering names; admittance ducts along
every axis equal the exact 1D solution).
"""
import numpy as np


def node_id(mesh, i, j, l):
    return i + (mesh.nx + 1) * (j + (mesh.ny + 1) * l)


def coords(mesh):
    """(n,3) node coordinates."""
    n = mesh.n_nodes
    ids = np.arange(n)
    i = ids % (mesh.nx + 1)
    j = (ids // (mesh.nx + 1)) % (mesh.ny + 1)
    l = ids // ((mesh.nx + 1) * (mesh.ny + 1))
    return np.stack([i * mesh.Lx / mesh.nx, j * mesh.Ly / mesh.ny, l * mesh.Lz / mesh.nz], axis=1)


def bricks(mesh):
    """(ne,8) vertex ids of every brick, local vertex a + 2b + 4c (bricks x fastest)."""
    I, J, L = np.meshgrid(np.arange(mesh.nx), np.arange(mesh.ny), np.arange(mesh.nz), indexing="ij")
    I, J, L = (A.transpose(2, 1, 0).ravel() for A in (I, J, L))  # l outer, i inner
    cols = [node_id(mesh, I + a, J + b, L + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    return np.stack(cols, axis=1).astype(np.int64)


def boundary_quads(mesh):
    """List of (4 vertex ids, (h_u, h_v)) per boundary quad in the documented order.

    Vertex order inside a quad: (u,v) in {(0,0),(1,0),(0,1),(1,1)}, u the first remaining axis.
    """
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    hx, hy, hz = mesh.Lx / nx, mesh.Ly / ny, mesh.Lz / nz
    quads = []
    # x- and x+ : (u,v) = (j,l)
    for i in (0, nx):
        for l in range(nz):
            for j in range(ny):
                quads.append(([node_id(mesh, i, j + du, l + dv) for dv in (0, 1) for du in (0, 1)], (hy, hz)))
    # y- and y+ : (u,v) = (i,l)
    for j in (0, ny):
        for l in range(nz):
            for i in range(nx):
                quads.append(([node_id(mesh, i + du, j, l + dv) for dv in (0, 1) for du in (0, 1)], (hx, hz)))
    # z- and z+ : (u,v) = (i,j)
    for l in (0, nz):
        for j in range(ny):
            for i in range(nx):
                quads.append(([node_id(mesh, i + du, j + dv, l) for dv in (0, 1) for du in (0, 1)], (hx, hy)))
    return quads
