"""The seeded workload generators produce the sizes the workload description states (CPU only)."""
import numpy as np

import helm_inputs as hi


def test_box_and_cabin_sizes():
    w = hi.workload("box100")
    m = w.problems[0].mesh
    assert m.n_nodes == 4641 and m.nnz27 == 110593
    c = hi.cabin_problem(100, 56, 48)
    assert c.mesh.n_nodes == 282093 and c.mesh.nnz27 == 7376005
    assert len(c.dir_nodes) == 525                      # 25 x 21 sun-roof nodes at h = 0.025
    assert np.count_nonzero(c.beta) == 2688            # 48 x 56 seat quads
    b = c.beta[c.beta != 0]
    assert b.real.min() >= 0.01 and b.real.max() <= 0.2 and np.abs(b.imag).max() <= 0.05
    big = hi.Mesh(200, 112, 96, *hi.CABIN)
    assert big.n_nodes == 2203161 and big.nnz27 == 58533193


def test_sweep_lattices():
    f = hi.sweep_freqs(256)
    dims = [hi.sweep_mesh_dims(x) for x in f]
    assert dims[0] == (24, 14, 12) and dims[-1] == (148, 83, 71)
    nodes = [(a + 1) * (b + 1) * (c + 1) for a, b, c in dims]
    assert nodes[-1] == 901152 and nodes[0] == 4875
    assert abs(sum(nodes) - 25.17e6) < 0.01e6
    assert sum(1 for d in dims if d == (24, 14, 12)) == 112


def test_boundary_numbering_and_draws_are_seeded():
    m = hi.Mesh(4, 3, 2, 1.0, 0.8, 0.6)
    off = m.side_offsets()
    assert off == [0, 6, 12, 20, 28, 40, 52] and m.n_bfaces == 52
    assert hi.floor_face_index(m, np.array([3]), np.array([2]))[0] == 28 + 3 + 4 * 2
    p1 = hi.cabin_problem(24, 14, 12)
    p2 = hi.cabin_problem(24, 14, 12)
    assert np.array_equal(p1.beta, p2.beta) and np.array_equal(p1.p_dir, p2.p_dir)
    w = hi.listener_weights(hi.Mesh(100, 56, 48, *hi.CABIN))
    assert abs(w.sum() - 1.0) < 1e-12 and (w > 0).sum() > 100


def test_resonance_sweep_inputs():
    f = hi.resonance_freqs(64)
    # bins 4..67 of a 512-point FFT at 256 Hz: spacing fs / N = 0.5 Hz
    assert np.allclose(np.diff(f), 256.0 / 512.0) and f[0] == 2.0 and f[-1] == 33.5
    a = hi.resonance_spectrum(f)
    assert f[np.argmax(np.abs(a))] == 13.0
    # the half-harmonic bump: a local maximum of |a| at 6.5 Hz
    k = int(np.where(f == 6.5)[0][0])
    assert abs(a[k]) > abs(a[k - 1]) and abs(a[k]) > abs(a[k + 1])
    # seeded: the same draw every time
    assert np.array_equal(a, hi.resonance_spectrum(f))
