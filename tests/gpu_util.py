"""Helpers for the GPU parity tests (marshalling only)."""
import numpy as np
import scipy.sparse as sp
import torch

from paper_2112_00087_gb300 import helm


def context(prob):
    m = prob.mesh
    ctx = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz, prob.c, prob.rho)
    nd = len(prob.dir_nodes)
    ctx.set_boundary(torch.from_numpy(prob.beta).cuda(),
                     torch.from_numpy(prob.dir_nodes.astype(np.int32)).cuda() if nd else None,
                     torch.from_numpy(prob.p_dir).cuda() if nd else None)
    return ctx


def gpu_matrix(ctx, freq, precision=helm.HELM_C128):
    A = helm.helm_assemble(ctx, freq, precision)
    rowptr, col, val = A.csr()
    n = ctx.n
    S = sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), rowptr.cpu().numpy()), shape=(n, n))
    return A, S, A.rhs.cpu().numpy() if A.rhs is not None else None


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dia_to_scipy(val27, mesh):
    """Slot-major [27, n] values -> scipy CSR (zero slots dropped), slot k = (di+1)+3(dj+1)+9(dl+1)."""
    v = val27.cpu().numpy()
    n = v.shape[1]
    Nx, Ny = mesh.nx + 1, mesh.ny + 1
    rows, cols, vals = [], [], []
    r = np.arange(n)
    for k in range(27):
        di, dj, dl = k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1
        c = r + di + Nx * (dj + Ny * dl)
        m = v[k] != 0
        rows.append(r[m]); cols.append(c[m]); vals.append(v[k][m])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
