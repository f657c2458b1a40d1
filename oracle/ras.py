"""Restricted additive Schwarz preconditioner (oracle; test infrastructure).

Paper Sec. 4 turns to overlapping Schwarz domain decomposition once one system no longer
fits one device. The oracle states the restricted additive Schwarz (RAS) preconditioner
used with GMRES:

  z = sum_s  Rt_s^T  A_s^{-1}  R_s r,   A_s = R_s A R_s^T,

where R_s restricts to subdomain s extended by ``overlap`` lattice layers and Rt_s keeps
only the nodes subdomain s owns (the owned sets partition the nodes). Ownership reading:
node (i,j,l) belongs to block (floor(i Px/(nx+1)), floor(j Py/(ny+1)), floor(l Pz/(nz+1)));
the extension is every node within Chebyshev index distance ``overlap`` of the owned box,
clamped to the lattice (the 27-point graph distance). Artificial boundaries are
homogeneous Dirichlet (A_s is the plain principal submatrix). Local solves are exact
(scipy splu).

Optimized Schwarz variant (``robin``; paper Sec. 4 names an optimized Schwarz method with
absorbing, Robin-type transmission conditions on the subdomain interfaces but gives no
parameters): A_s = R_s A R_s^T + robin * M_G,s, where M_G,s is the face mass (int Ni Nj dS, the
same Q1 face integral as the admittance term) of every face of the extended box that lies inside
the lattice (an artificial interface), restricted to nodes that are not Dirichlet nodes. Reading
of the coefficient: robin = i k, the matched impedance (beta rho c = 1) of the wall term
+ i k rho c B(beta) of the operator, i.e. the first-order absorbing (Despres) condition, the same
on both sides of an interface.

Two-sided variant (``robin=(c_lo, c_hi)``; the paper's optimized Schwarz method uses two-sided
interface conditions, i.e. different conditions on the two sides of an interface, and again gives
no parameters): A_s = R_s A R_s^T + sum over the artificial faces of the extended box of
(c / h_a) M_face, c = c_lo on the box's low faces (the plane i = i0, j = j0 or l = l0) and c = c_hi
on its high faces, h_a the lattice spacing normal to the face (a plane that is both, in a box one
layer thick, takes c_lo). Across an interface the subdomain below sees c_hi and the one above c_lo.
The coefficients are dimensionless; the reading of their values (a discrete optimisation of the
pair on a small cabin) is stated where they are used.

Pinned (tests/test_oracle_ras.py): a 1x1x1 partition is the exact inverse (GMRES converges
in one step); with any partition the preconditioned solution equals the direct solution; the
interface mass of a box equals the scatter of fem.quad_mass over the box's interface quads.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import fem


def block_ranges(npts, parts):
    """Owned index ranges [lo, hi) along one axis: point t goes to floor(t*parts/npts)."""
    owner = (np.arange(npts) * parts) // npts
    return [(int(np.argmax(owner == p)), int(npts - np.argmax(owner[::-1] == p))) for p in range(parts)]


def subdomains(mesh, parts=(8, 4, 4), overlap=2):
    """List of (owned_box, extended_box) with boxes ((i0,i1),(j0,j1),(l0,l1)), half-open."""
    dims = (mesh.nx + 1, mesh.ny + 1, mesh.nz + 1)
    rngs = [block_ranges(d, p) for d, p in zip(dims, parts)]
    out = []
    for bl in range(parts[2]):
        for bj in range(parts[1]):
            for bi in range(parts[0]):
                own = (rngs[0][bi], rngs[1][bj], rngs[2][bl])
                ext = tuple((max(0, lo - overlap), min(d, hi + overlap)) for (lo, hi), d in zip(own, dims))
                out.append((own, ext))
    return out


def _box_ids(mesh, box):
    (i0, i1), (j0, j1), (l0, l1) = box
    i, j, l = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), np.arange(l0, l1), indexing="ij")
    ids = i + (mesh.nx + 1) * (j + (mesh.ny + 1) * l)
    return np.sort(ids.ravel())


def interface_mass(mesh, ext, side="both", scaled=False):
    """Face mass (n x n real CSR) of the faces of box ``ext`` that lie inside the lattice: the
    scatter of fem.quad_mass over every quad of those faces. side: "both", "lo" (the planes
    i0, j0, l0) or "hi" (the planes i1-1, j1-1, l1-1, except one that is also a low plane).
    scaled: each face's mass divided by the lattice spacing normal to it."""
    dims = (mesh.nx + 1, mesh.ny + 1, mesh.nz + 1)
    h = (mesh.Lx / mesh.nx, mesh.Ly / mesh.ny, mesh.Lz / mesh.nz)
    rows, cols, vals = [], [], []
    for a in range(3):
        (lo, hi) = ext[a]
        planes = []
        if side in ("both", "lo") and lo > 0:
            planes.append(lo)
        if side in ("both", "hi") and hi < dims[a] and not (side == "hi" and lo > 0 and hi - 1 == lo):
            planes.append(hi - 1)
        u, v = [b for b in range(3) if b != a]
        Bq = fem.quad_mass(h[u], h[v]) / (h[a] if scaled else 1.0)
        for pa in sorted(set(planes)):
            for cu in range(ext[u][0], ext[u][1] - 1):
                for cv in range(ext[v][0], ext[v][1] - 1):
                    ids = []
                    for b2 in (0, 1):
                        for b1 in (0, 1):
                            idx = [0, 0, 0]
                            idx[a], idx[u], idx[v] = pa, cu + b1, cv + b2
                            ids.append(idx[0] + dims[0] * (idx[1] + dims[1] * idx[2]))
                    for r in range(4):
                        for c in range(4):
                            rows.append(ids[r]); cols.append(ids[c]); vals.append(Bq[r, c])
    n = dims[0] * dims[1] * dims[2]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


class RAS:
    def __init__(self, A, mesh, parts=(8, 4, 4), overlap=2, robin=None, dir_nodes=None):
        A = A.tocsr()
        self.n = A.shape[0]
        self.blocks = []
        free = np.ones(self.n, dtype=bool)
        if dir_nodes is not None:
            free[np.asarray(dir_nodes)] = False
        for own, ext in subdomains(mesh, parts, overlap):
            E = _box_ids(mesh, ext)
            O = _box_ids(mesh, own)
            keep = np.searchsorted(E, O)  # positions of owned nodes inside E
            As = A[E][:, E]
            if robin is not None:
                F = sp.diags(free[E].astype(np.float64))
                if np.ndim(robin) == 0:
                    As = As + robin * (F @ interface_mass(mesh, ext)[E][:, E] @ F)
                else:  # two-sided: dimensionless (c_lo, c_hi), per face times 1 / h_normal
                    for c, side in zip(robin, ("lo", "hi")):
                        As = As + c * (F @ interface_mass(mesh, ext, side, scaled=True)[E][:, E] @ F)
            lu = spl.splu(As.tocsc())
            self.blocks.append((E, O, keep, lu))

    def __call__(self, r):
        z = np.zeros(self.n, dtype=np.complex128)
        for E, O, keep, lu in self.blocks:
            zE = lu.solve(np.asarray(r[E], dtype=np.complex128))
            z[O] = zE[keep]
        return z
