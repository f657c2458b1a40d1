"""Listener objective and its adjoint gradient (oracle; test infrastructure).

J = sum_f sum_i w_i |p_i(f)|^2 with w_i = 1/|S| on the listener nodes S (mean square
pressure), p(f) the frequency response of the cavity problem (paper Sec. 3.2).

Derivation (PyTorch convention for a real loss of complex inputs: grad = dJ/dRe + i dJ/dIm):
with A_red p = b (A_red complex symmetric after symmetric Dirichlet elimination), solve the
adjoint system A_red lam = W conj(p). Zero lam on the Dirichlet nodes to get lam_F. Then

  per boundary quad e:   g_e = lam_F^T (i k rho c B_e) p,   grad_beta_e = -2 conj(g_e)
  per Dirichlet node:    mu = W_D conj(p_D) - A_DF lam_F,     grad_p_D    =  2 conj(mu)

with B_e the quad mass of face e and A_DF taken from the matrix before elimination; both
summed over frequencies. Solves use scipy's sparse LU, or with ``dense=True`` a dense LU of the
full matrix (LAPACK getrf/getrs through scipy.linalg) -- the plain definition of the solve, for
lattices small enough to hold A densely (config 0's 4,641 nodes: 344 MB).

Pinned (tests/test_oracle_adjoint.py): central finite differences of J (perturbing real and
imaginary parts separately) on random faces and Dirichlet nodes.
"""
import numpy as np
import scipy.sparse.linalg as spl

from . import fem, mesh as _mesh


def objective_and_gradient(prob, freqs, w, KM=None, dense=False):
    """Returns (J, grad_beta [n_bfaces] complex, grad_pdir [n_dir] complex, list of p)."""
    m = prob.mesh
    KM = KM if KM is not None else fem.assemble_KM(m)
    quads = _mesh.boundary_quads(m)
    Bq = {}
    J = 0.0
    gb = np.zeros(m.n_bfaces, dtype=np.complex128)
    gd = np.zeros(len(prob.dir_nodes), dtype=np.complex128)
    isD = np.zeros(m.n_nodes, dtype=bool)
    isD[prob.dir_nodes] = True
    ps = []
    for f in freqs:
        A = fem.helmholtz_matrix(prob, f, KM)
        A_red, b = fem.eliminate_dirichlet(A, prob.dir_nodes, prob.p_dir)
        if dense:
            import scipy.linalg as sla
            lu = sla.lu_factor(A_red.toarray())
            solve = lambda v: sla.lu_solve(lu, v)  # noqa: E731
        else:
            lu = spl.splu(A_red.tocsc())
            solve = lu.solve
        p = solve(b)
        ps.append(p)
        J += float(np.sum(w * np.abs(p) ** 2))
        lam = solve(w * np.conj(p))
        lamF = np.where(isD, 0.0, lam)
        k = fem.wavenumber(f, prob.c)
        for e, (nodes, (hu, hv)) in enumerate(quads):
            key = (hu, hv)
            if key not in Bq:
                Bq[key] = fem.quad_mass(hu, hv)
            nodes = np.asarray(nodes)
            g = 1j * k * prob.rho * prob.c * (lamF[nodes] @ Bq[key] @ p[nodes])
            gb[e] += -2.0 * np.conj(g)
        mu = w[prob.dir_nodes] * np.conj(p[prob.dir_nodes]) - A[prob.dir_nodes] @ lamF
        gd += 2.0 * np.conj(mu)
    return J, gb, gd, ps


def objective(prob, freqs, w, KM=None):
    """J alone (direct solves), used for finite differences."""
    KM = KM if KM is not None else fem.assemble_KM(prob.mesh)
    J = 0.0
    for f in freqs:
        A_red, b = fem.system(prob, f, KM)
        p = spl.spsolve(A_red.tocsc(), b)
        J += float(np.sum(w * np.abs(p) ** 2))
    return J
