"""Pins for the oracle's submatrix matrix functions (oracle/functions.py): A^-1/2, A^1/2, A^-1.

Each check is independent of the oracle's eigendecomposition formula: a diagonal input
(elementwise powers), the dense function of a full pattern from numpy's eigh of the whole
matrix, the identity F A F = I, block-diagonal inputs and an independent iteration.
"""

import numpy as np
import pytest

import oracle as O
from synth import make_lattice_system, make_overlap_system


def _system(r_c, n_mol=16, seed=5):
    return make_overlap_system(n_mol, 4, r_c, 1.5, seed)


def test_overlap_generator_is_positive_definite():
    s = _system(6.0, n_mol=64)
    a = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    lo, _ = O.gershgorin_bounds(a)
    assert lo > 0.3 and np.allclose(a, a.T)


POWER = {"inv_sqrt": -0.5, "sqrt": 0.5, "inv": -1.0}


@pytest.mark.parametrize("f", ["inv_sqrt", "sqrt", "inv"])
def test_diagonal_blocks_elementwise(f):
    # block-diagonal with diagonal blocks: f is the elementwise power
    s = make_lattice_system(8, 3, 0.0, 1.5, 9)  # cutoff 0: diagonal blocks only
    d = np.abs(np.random.default_rng(1).normal(1.0, 0.3, 24)) + 0.2
    vals = np.zeros_like(s.values)
    for j in range(8):
        blk = np.diag(d[3 * j:3 * j + 3])
        vals[9 * j:9 * j + 9] = blk.T.reshape(-1)
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, vals, f)
    p = POWER[f]
    ref = np.zeros_like(vals)
    for j in range(8):
        ref[9 * j:9 * j + 9] = np.diag(d[3 * j:3 * j + 3] ** p).T.reshape(-1)
    assert np.max(np.abs(res.values - ref)) < 1e-14
    assert abs(res.trace - np.sum(d ** p)) < 1e-12


@pytest.mark.parametrize("f", ["inv_sqrt", "sqrt", "inv"])
def test_full_pattern_equals_dense_function(f):
    s = _system(np.inf)
    a = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    lam, v = np.linalg.eigh(a)
    dense = (v * (lam ** POWER[f])) @ v.T
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, f)
    got = O.to_dense(s.block_size, s.col_ptr, s.row_idx, res.values)
    assert np.max(np.abs(got - dense)) < 1e-12
    if f == "inv_sqrt":
        assert np.max(np.abs(got @ a @ got - np.eye(a.shape[0]))) < 1e-12
    if f == "inv":
        assert np.max(np.abs(got @ a - np.eye(a.shape[0]))) < 1e-12
        assert np.max(np.abs(got - np.linalg.solve(a, np.eye(a.shape[0])))) < 1e-12


def test_block_diagonal_is_exact():
    s = _system(0.0)  # cutoff 0: every block column is its own submatrix
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, "inv_sqrt")
    for j in range(s.block_size.shape[0]):
        a = s.values[16 * j:16 * j + 16].reshape(4, 4).T
        w, v = np.linalg.eigh(a)
        ref = (v / np.sqrt(w)) @ v.T
        assert np.max(np.abs(res.values[16 * j:16 * j + 16].reshape(4, 4).T - ref)) < 1e-14


@pytest.mark.parametrize("n", [3, 12, 40])
def test_eig_matches_coupled_newton_schulz(n):
    rng = np.random.default_rng(n)
    g = rng.normal(size=(n, n))
    a = g @ g.T / n + np.eye(n)
    c = float(np.max(np.sum(np.abs(a), axis=1)))  # Gershgorin: c >= rho(A)
    root, iroot = O.coupled_newton_schulz(a, c)
    assert np.max(np.abs(root - O.apply_eig(a, "sqrt"))) < 1e-12
    assert np.max(np.abs(iroot - O.apply_eig(a, "inv_sqrt"))) < 1e-12


def test_submatrix_columns_differ_from_dense_when_truncated():
    # the method is an approximation: with a cutoff the result departs from the dense function,
    # by less than the dropped couplings
    s = _system(5.0, n_mol=27)
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, "inv_sqrt")
    a = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    lam, v = np.linalg.eigh(a)
    dense = (v / np.sqrt(lam)) @ v.T
    got = O.to_dense(s.block_size, s.col_ptr, s.row_idx, res.values)
    mask = got != 0.0
    err = np.max(np.abs((got - dense)[mask]))
    assert 1e-8 < err < 5e-2
