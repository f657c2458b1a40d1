"""Pin of the oracle's adjoint gradient by central finite differences (CPU only)."""
import numpy as np

import helm_inputs as hi
from oracle import adjoint, fem


def small_cabin():
    # cabin-shaped 2.5 x 1.4 x 1.2 box on a coarse lattice, with the sun-roof patch and the
    # seat admittances of the full-size workloads
    return hi.cabin_problem(10, 7, 6, beta_seed=1, p_scale=0.1)


def test_adjoint_gradient_matches_central_differences():
    prob = small_cabin()
    m = prob.mesh
    w = hi.listener_weights(m, centre=(1.6, 0.4, 0.9), radius=0.45)
    assert (w > 0).sum() > 0
    freqs = [60.0, 110.0]
    KM = fem.assemble_KM(m)
    J, gb, gd, _ = adjoint.objective_and_gradient(prob, freqs, w, KM)
    rng = np.random.default_rng(0)
    faces = rng.choice(np.flatnonzero(prob.beta != 0), 8, replace=False)
    faces = np.concatenate([faces, rng.choice(m.n_bfaces, 4, replace=False)])  # rigid ones too
    h = 1e-6
    for e in faces:
        for unit in (1.0, 1j):
            bp, bm = prob.beta.copy(), prob.beta.copy()
            bp[e] += h * unit
            bm[e] -= h * unit
            Jp = adjoint.objective(hi.Problem(m, bp, prob.dir_nodes, prob.p_dir), freqs, w, KM)
            Jm = adjoint.objective(hi.Problem(m, bm, prob.dir_nodes, prob.p_dir), freqs, w, KM)
            fd = (Jp - Jm) / (2 * h)
            an = gb[e].real if unit == 1.0 else gb[e].imag
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-3 * np.abs(gb).max())
    for t in rng.choice(len(prob.dir_nodes), 5, replace=False):
        for unit in (1.0, 1j):
            pp, pm = prob.p_dir.copy(), prob.p_dir.copy()
            pp[t] += h * unit
            pm[t] -= h * unit
            Jp = adjoint.objective(hi.Problem(m, prob.beta, prob.dir_nodes, pp), freqs, w, KM)
            Jm = adjoint.objective(hi.Problem(m, prob.beta, prob.dir_nodes, pm), freqs, w, KM)
            fd = (Jp - Jm) / (2 * h)
            an = gd[t].real if unit == 1.0 else gd[t].imag
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-3 * np.abs(gd).max())


def test_dense_and_sparse_adjoints_agree():
    # the dense LU form (the plain definition of the solves) and the sparse LU form give the same
    # objective and gradients to rounding
    prob = hi.small_box_problem(8, 6, 5)
    w = hi.listener_weights(prob.mesh, centre=(0.5, 0.4, 0.3), radius=0.2)
    J1, gb1, gd1, _ = adjoint.objective_and_gradient(prob, [100.0, 170.0], w)
    J2, gb2, gd2, _ = adjoint.objective_and_gradient(prob, [100.0, 170.0], w, dense=True)
    assert abs(J1 - J2) <= 1e-12 * J1
    assert np.linalg.norm(gb1 - gb2) <= 1e-11 * np.linalg.norm(gb1)
    assert np.linalg.norm(gd1 - gd2) <= 1e-11 * np.linalg.norm(gd1)
