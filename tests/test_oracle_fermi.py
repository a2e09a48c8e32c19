"""Pins of the finite-temperature Fermi oracle (oracle/fermi.py) against facts that do not go
through its eigendecomposition formula: the logistic function on diagonal inputs, the
zero-temperature limit (the density-matrix oracle), a dense matrix exponential on a full
pattern, particle-hole symmetry per block column, the infinite-temperature limit and the
monotone trace."""

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from oracle.fermi import fermi_submatrix
from synth import make_lattice_system


def _system(r_c, n_mol=16, seed=5):
    return make_lattice_system(n_mol, 6, r_c, 1.5, seed)


def test_diagonal_inputs_are_the_logistic_function():
    s = make_lattice_system(8, 3, 0.0, 1.5, 9)  # cutoff 0: diagonal blocks only
    d = np.random.default_rng(1).normal(0.0, 0.5, 24)
    vals = np.zeros_like(s.values)
    for j in range(8):
        vals[9 * j:9 * j + 9] = np.diag(d[3 * j:3 * j + 3]).T.reshape(-1)
    mu, beta = 0.1, 7.0
    res = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, vals, mu, beta)
    occ = 1.0 / (1.0 + np.exp(beta * (d - mu)))
    ref = np.zeros_like(vals)
    for j in range(8):
        ref[9 * j:9 * j + 9] = np.diag(occ[3 * j:3 * j + 3]).T.reshape(-1)
    assert np.max(np.abs(res.values - ref)) < 1e-15
    assert abs(res.trace - occ.sum()) < 1e-13


def test_zero_temperature_limit_is_the_density_matrix():
    s = _system(4.5)
    d = O.density_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.0)
    assert np.min(d.min_abs_eig) > 0.05  # mu = 0 in a gap of every submatrix
    f = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.0, 2e3)
    assert np.max(np.abs(f.values - d.values)) < 1e-12
    assert abs(f.trace - d.trace) < 1e-10


@pytest.mark.parametrize("mu,beta", [(0.0, 4.0), (0.2, 20.0), (-0.4, 1.0)])
def test_full_pattern_against_the_matrix_exponential(mu, beta):
    s = _system(np.inf, n_mol=8)
    h = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    n = h.shape[0]
    ref = np.linalg.solve(np.eye(n) + scipy.linalg.expm(beta * (h - mu * np.eye(n))), np.eye(n))
    res = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, mu, beta)
    got = O.to_dense(s.block_size, s.col_ptr, s.row_idx, res.values)
    assert np.max(np.abs(got - ref)) < 1e-11
    assert np.max(np.abs(got @ h - h @ got)) < 1e-11  # a function of H commutes with H


def test_particle_hole_symmetry_per_block_column():
    # f(2 mu - x) = 1 - f(x), and T_j(2 mu I - H) = 2 mu I - T_j(H) on the same pattern, so the
    # owner columns satisfy F'[R_j, j] = E_j - F[R_j, j] even on a truncated pattern
    s = _system(4.5, n_mol=27)
    mu, beta = 0.05, 6.0
    off = O.block_value_offsets(s.block_size, s.col_ptr, s.row_idx)
    mirrored = -s.values.copy()
    eye = np.zeros_like(s.values)
    for j in range(s.n_blocks):
        for k in range(s.col_ptr[j], s.col_ptr[j + 1]):
            if s.row_idx[k] == j:
                mirrored[off[k]:off[k + 1]] += 2.0 * mu * np.eye(6).reshape(-1)
                eye[off[k]:off[k + 1]] = np.eye(6).reshape(-1)
    f = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, mu, beta)
    g = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, mirrored, mu, beta)
    assert np.max(np.abs(f.values + g.values - eye)) < 1e-13
    assert abs(f.trace + g.trace - s.n) < 1e-11


def test_infinite_temperature_limit_and_monotone_trace():
    s = _system(4.5)
    f0 = fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.0, 0.0)
    off = O.block_value_offsets(s.block_size, s.col_ptr, s.row_idx)
    half = np.zeros_like(s.values)
    for j in range(s.n_blocks):
        for k in range(s.col_ptr[j], s.col_ptr[j + 1]):
            if s.row_idx[k] == j:
                half[off[k]:off[k + 1]] = 0.5 * np.eye(6).reshape(-1)
    assert np.max(np.abs(f0.values - half)) < 1e-14
    traces = [fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, mu, 8.0).trace
              for mu in np.linspace(-1.0, 1.0, 9)]
    assert all(a < b for a, b in zip(traces, traces[1:]))
    assert traces[0] < 0.05 * s.n and traces[-1] > 0.95 * s.n
