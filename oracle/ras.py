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

Pinned (tests/test_oracle_ras.py): a 1x1x1 partition is the exact inverse (GMRES converges
in one step); with any partition the preconditioned solution equals the direct solution.
"""
import numpy as np
import scipy.sparse.linalg as spl


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


class RAS:
    def __init__(self, A, mesh, parts=(8, 4, 4), overlap=2):
        A = A.tocsr()
        self.n = A.shape[0]
        self.blocks = []
        for own, ext in subdomains(mesh, parts, overlap):
            E = _box_ids(mesh, ext)
            O = _box_ids(mesh, own)
            keep = np.searchsorted(E, O)  # positions of owned nodes inside E
            lu = spl.splu(A[E][:, E].tocsc())
            self.blocks.append((E, O, keep, lu))

    def __call__(self, r):
        z = np.zeros(self.n, dtype=np.complex128)
        for E, O, keep, lu in self.blocks:
            zE = lu.solve(np.asarray(r[E], dtype=np.complex128))
            z[O] = zE[keep]
        return z
