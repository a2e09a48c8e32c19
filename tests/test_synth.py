"""The seeded generators: shapes, symmetry, determinism, distributions."""

import numpy as np

import oracle as O
from synth import keyed_normals, make_lattice_system, make_workload, md_trajectory, spectrum_matrix


def test_lattice_system_shapes_and_symmetry():
    s = make_workload("water32")
    assert s.n_blocks == 32 and s.n == 192 and s.n_occ == 96
    assert abs(s.box[0] - 3.1 * 32 ** (1 / 3)) < 1e-12
    a = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    assert np.array_equal(a, a.T)
    for j in range(s.n_blocks):  # sorted rows, diagonal present
        rows = s.row_idx[s.col_ptr[j]:s.col_ptr[j + 1]]
        assert np.all(np.diff(rows) > 0) and j in rows


def test_generator_is_deterministic_and_keyed():
    a = make_workload("water32")
    b = make_workload("water32")
    assert np.array_equal(a.values, b.values) and np.array_equal(a.row_idx, b.row_idx)
    x = keyed_normals(5, np.array([1, 2]), np.array([3, 4]), 10)
    y = keyed_normals(5, np.array([2]), np.array([4]), 10)
    assert np.array_equal(x[1], y[0])
    z = keyed_normals(7, np.arange(2000), np.arange(2000) + 1, 50).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_diagonal_block_bands():
    s = make_lattice_system(64, 6, r_c=0.01, ell=1.5, seed=3)
    lam = np.linalg.eigvalsh(O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values))
    assert np.count_nonzero(lam < 0) == 64 * 3
    assert abs(np.mean(lam[lam < 0]) + 0.5) < 0.02 and abs(np.mean(lam[lam > 0]) - 0.5) < 0.02


def test_trajectory_pattern_changes_smoothly():
    snaps = list(md_trajectory(64, 6, 6.0, 1.5, seed=4, n_snap=3))
    assert len(snaps) == 3
    d = [O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values) for s in snaps]
    assert 0 < np.max(np.abs(d[1] - d[0])) < 0.05


def test_spectrum_matrix():
    a = spectrum_matrix(20, np.linspace(-1, 1, 20), seed=1)
    assert np.allclose(np.linalg.eigvalsh(a), np.linspace(-1, 1, 20), atol=1e-13)


def test_nonorth_pair_shares_the_pattern_and_s_is_positive_definite():
    from synth import make_nonorth_pair

    h, s = make_nonorth_pair(64, 6, 6.0, 1.5, 11)
    assert np.array_equal(h.col_ptr, s.col_ptr) and np.array_equal(h.row_idx, s.row_idx)
    hd = O.to_dense(h.block_size, h.col_ptr, h.row_idx, h.values)
    sd = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    assert np.allclose(hd, hd.T) and np.allclose(sd, sd.T)
    lo, _ = O.gershgorin_bounds(sd)
    assert lo > 0.1  # every Gershgorin disc of S well right of zero
    # S's off-diagonal blocks come from their own key stream, not from H's
    off = ~np.eye(hd.shape[0], dtype=bool) & (hd != 0)
    assert abs(np.corrcoef(hd[off], sd[off])[0, 1]) < 0.1
    h2, s2 = make_nonorth_pair(64, 6, 6.0, 1.5, 11)
    assert np.array_equal(h.values, h2.values) and np.array_equal(s.values, s2.values)
