"""Pins of the non-orthogonal oracle (Eq. 14 with S != I, oracle/nonorth.py) against facts
that do not go through its own formula: the orthogonal oracle at S = I, the dense Loewdin
form and the inertia of H - mu S on a full pattern, congruence with a block-diagonal
basis change, and the end points of the bracket."""

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from synth import make_nonorth_pair


def _pair(n_mol=12, r_c=5.0, seed=3):
    return make_nonorth_pair(n_mol, 6, r_c, 1.5, seed)


def test_identity_overlap_gives_the_orthogonal_oracle():
    h, _ = _pair(r_c=4.0)
    s_vals = np.zeros_like(h.values)
    off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
    for j in range(h.n_blocks):
        for k in range(h.col_ptr[j], h.col_ptr[j + 1]):
            if h.row_idx[k] == j:
                s_vals[off[k]:off[k + 1]] = np.eye(6).reshape(-1)
    for mu in (-0.3, 0.0, 0.2):
        p = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s_vals, mu)
        d = O.density_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, mu)
        assert np.max(np.abs(p.values - d.values)) <= 1e-12
        assert abs(p.trace - d.trace) <= 1e-11 and abs(p.energy - d.energy) <= 1e-11


def _dense_inertia_below(h, s, mu):
    """Number of eigenvalues of the pencil (h, s) below mu: the negative inertia of h - mu s
    from an LDL^T factorisation (Sylvester's law of inertia)."""
    _, dblk, _ = scipy.linalg.ldl(h - mu * s)
    return int(np.count_nonzero(np.linalg.eigvalsh(dblk) < 0))


@pytest.mark.parametrize("mu", [-0.2, 0.05, 0.3])
def test_full_pattern_is_the_dense_loewdin_projector(mu):
    h, s = _pair(n_mol=8, r_c=np.inf, seed=5)
    assert np.all(np.diff(h.col_ptr) == h.n_blocks)  # one submatrix = the whole matrix
    p = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, mu)
    hd = O.to_dense(h.block_size, h.col_ptr, h.row_idx, h.values)
    sd = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    pd = O.to_dense(h.block_size, h.col_ptr, h.row_idx, p.values)
    # Loewdin: S^-1/2 D(S^-1/2 H S^-1/2) S^-1/2 with the orthogonal projector D
    lam, v = np.linalg.eigh(sd)
    li = (v * lam ** -0.5) @ v.T
    ref = li @ O.dense_density(li @ hd @ li, mu) @ li
    assert np.max(np.abs(pd - ref)) <= 1e-12
    # idempotent in the S metric; tr(P S) counts the pencil's eigenvalues below mu
    assert np.max(np.abs(pd @ sd @ pd - pd)) <= 1e-12
    n_below = _dense_inertia_below(hd, sd, mu)
    assert abs(p.trace - n_below) <= 1e-10
    assert abs(np.trace(pd @ sd) - n_below) <= 1e-10
    assert abs(p.energy - np.trace(pd @ hd)) <= 1e-10


def test_congruence_with_a_block_diagonal_basis_change():
    # H' = C^T H C, S' = C^T S C with block-diagonal invertible C keep the pattern, and
    # P'[r, j] = C_r^-1 P[r, j] C_j^-T block by block (also for the submatrix method)
    h, s = _pair(n_mol=16, r_c=4.5, seed=9)
    rng = np.random.default_rng(2)
    cb = np.eye(6)[None] + 0.2 * rng.standard_normal((h.n_blocks, 6, 6))
    off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)

    def transform(vals):
        out = np.empty_like(vals)
        for j in range(h.n_blocks):
            for k in range(h.col_ptr[j], h.col_ptr[j + 1]):
                r = h.row_idx[k]
                blk = vals[off[k]:off[k + 1]].reshape(6, 6).T
                out[off[k]:off[k + 1]] = (cb[r].T @ blk @ cb[j]).T.reshape(-1)
        return out

    mu = 0.0
    p = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, mu)
    p2 = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, transform(h.values), transform(s.values), mu)
    err = 0.0
    for j in range(h.n_blocks):
        for k in range(h.col_ptr[j], h.col_ptr[j + 1]):
            r = h.row_idx[k]
            blk = p.values[off[k]:off[k + 1]].reshape(6, 6).T
            want = np.linalg.solve(cb[r], blk) @ np.linalg.inv(cb[j]).T
            got = p2.values[off[k]:off[k + 1]].reshape(6, 6).T
            err = max(err, float(np.max(np.abs(got - want))))
    assert err <= 1e-11
    assert abs(p2.trace - p.trace) <= 1e-10  # tr(P S) is invariant


def test_scaling_the_pair():
    h, s = _pair(seed=4)
    p = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, 0.1)
    p2 = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, 2.0 * h.values, 2.0 * s.values, 0.1)
    assert np.max(np.abs(p2.values - 0.5 * p.values)) <= 1e-13


def test_bracket_end_points():
    h, s = _pair(n_mol=16, r_c=4.5, seed=6)
    lo, hi = O.nonorth_bracket(h.block_size, h.col_ptr, h.row_idx, h.values, s.values)
    below = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, lo - 1e-9)
    above = O.density_nonorth_submatrix(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, hi + 1e-9)
    assert np.max(np.abs(below.values)) <= 1e-12 and abs(below.trace) <= 1e-12
    assert abs(above.trace - h.n) <= 1e-10  # P_j = A_S^-1 for every j
    assert lo < -0.3 and hi > 0.3  # both bands inside


def test_bisection_matches_the_electron_count():
    h, s = _pair(n_mol=16, r_c=4.5, seed=6)
    n_e = float(h.n // 2)
    # the submatrix trace is piecewise constant in mu with non-integer steps: a tolerance of 1/2
    mu, res, hist = O.bisect_mu_nonorth(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, n_e, 40, 0.5)
    assert abs(res.trace - n_e) <= 0.5
    assert hist[-1][0] == mu and len(hist) < 40
    traces = [t for _, t in sorted(hist)]
    assert all(a <= b + 1e-9 for a, b in zip(traces, traces[1:]))  # tr(P(mu) S) grows with mu


def test_take_blocks_follows_the_filter_flags():
    h, s = _pair(n_mol=64, r_c=6.0, seed=8)
    cp, ri, hv, keep = O.filter_blocks(h.block_size, h.col_ptr, h.row_idx, h.values, 2e-2)
    assert 0 < np.count_nonzero(~keep)
    sv = O.take_blocks(h.block_size, h.col_ptr, h.row_idx, s.values, keep)
    assert sv.shape == hv.shape
    off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
    foff = O.block_value_offsets(h.block_size, cp, ri)
    kk = np.flatnonzero(keep)
    for t in (0, len(kk) // 2, len(kk) - 1):
        k = kk[t]
        assert np.array_equal(sv[foff[t]:foff[t + 1]], s.values[off[k]:off[k + 1]])
