"""Pins for the oracle's submatrix method (Fig. 2) and purification (Eq. 14).

The method is exact when one submatrix is the whole matrix, or when the
matrix is block diagonal; a tiny brute-force implementation (dense indexing,
Newton sign iteration) checks the general case; trace/energy and the
bisection are checked against closed forms and monotonicity.
"""

import numpy as np
import pytest

import oracle as O
from synth import make_lattice_system, make_workload


def _filtered(s, eps=0.0):
    cp, ri, v, _ = O.filter_blocks(s.block_size, s.col_ptr, s.row_idx, s.values, eps)
    return s.block_size, cp, ri, v


def _hand_matrix():
    """3 block columns with block sizes (2, 1, 2); explicit values, column-major blocks."""
    bs = np.array([2, 1, 2], dtype=np.int32)
    # pattern: (0,0) (1,0) (2,0) | (0,1) (1,1) | (0,2) (2,2)
    col_ptr = np.array([0, 3, 5, 7], dtype=np.int64)
    row_idx = np.array([0, 1, 2, 0, 1, 0, 2], dtype=np.int32)
    h00 = np.array([[1.0, 0.5], [0.5, -1.0]])
    h10 = np.array([[0.3, -0.4]])  # 1x2, rows of block 1, cols of block 0
    h20 = np.array([[1e-4, 0.0], [0.0, 1e-4]])  # Frobenius norm 1.414e-4
    h11 = np.array([[0.2]])
    h22 = np.array([[0.0, 0.0], [0.0, 0.0]])  # a zero diagonal block
    blocks = [h00, h10, h20, h10.T, h11, h20.T, h22]
    values = np.concatenate([b.T.reshape(-1) for b in blocks])
    return bs, col_ptr, row_idx, values, dict(h00=h00, h10=h10, h20=h20, h11=h11, h22=h22)


def test_to_dense_column_major_blocks():
    bs, cp, ri, v, h = _hand_matrix()
    a = O.to_dense(bs, cp, ri, v)
    assert a.shape == (5, 5)
    assert np.array_equal(a[0:2, 0:2], h["h00"])
    assert np.array_equal(a[2:3, 0:2], h["h10"])
    assert np.array_equal(a[0:2, 2:3], h["h10"].T)
    assert np.array_equal(a[3:5, 0:2], h["h20"])
    assert a[2, 3] == 0.0 and a[3, 2] == 0.0  # block (2,1) absent
    assert np.array_equal(a, a.T)


def test_filter_rule_strict_and_diagonal_kept():
    bs, cp, ri, v, _ = _hand_matrix()
    norm20 = np.sqrt(2) * 1e-4
    # eps just above the norm of the (2,0)/(0,2) blocks drops them; the zero diagonal block stays
    cp2, ri2, v2, keep = O.filter_blocks(bs, cp, ri, v, norm20 * 1.000001)
    assert list(keep) == [True, True, False, True, True, False, True]
    assert list(cp2) == [0, 2, 4, 5] and list(ri2) == [0, 1, 0, 1, 2]
    # eps equal to the norm keeps them (strict "<" drops)
    _, _, _, keep = O.filter_blocks(bs, cp, ri, v, norm20)
    assert keep.all()
    # the filtered values are the surviving blocks, in order
    a2 = O.to_dense(bs, cp2, ri2, v2)
    a = O.to_dense(bs, cp, ri, v)
    a[3:5, 0:2] = 0.0
    a[0:2, 3:5] = 0.0
    assert np.array_equal(a2, a)


def test_gather_hand_matrix():
    bs, cp, ri, v, h = _hand_matrix()
    # column 1 keeps rows {0, 1}: T_1 = H[{0,1},{0,1}] - mu I
    t, rows, local = O.gather_submatrix(bs, cp, ri, v, 1, mu=0.25)
    assert list(rows) == [0, 1] and list(local) == [0, 2, 3]
    ref = np.zeros((3, 3))
    ref[0:2, 0:2] = h["h00"]
    ref[2:3, 0:2] = h["h10"]
    ref[0:2, 2:3] = h["h10"].T
    ref[2, 2] = 0.2
    assert np.array_equal(t, ref - 0.25 * np.eye(3))
    # column 0 keeps rows {0,1,2}; block (2,1) is absent from H so T_0[block 2, block 1] = 0
    t, rows, local = O.gather_submatrix(bs, cp, ri, v, 0, mu=0.0)
    assert list(rows) == [0, 1, 2]
    assert np.all(t[3:5, 2:3] == 0.0) and np.all(t[2:3, 3:5] == 0.0)
    assert np.array_equal(t[3:5, 0:2], h["h20"])


@pytest.mark.parametrize("mu", [0.0, 0.3, -0.45])
def test_full_pattern_equals_dense(mu):
    s = make_workload("water32_full")
    bs, cp, ri, v = _filtered(s)
    res = O.density_submatrix(bs, cp, ri, v, mu)
    d_sub = O.to_dense(bs, cp, ri, res.values)
    h = O.to_dense(bs, cp, ri, v)
    d_ref = O.dense_density(h, mu)
    assert np.max(np.abs(d_sub - d_ref)) < 1e-12
    lam = np.linalg.eigvalsh(h)
    # closed forms: trace = number of eigenvalues below mu, E = sum of those eigenvalues
    assert abs(res.trace - np.count_nonzero(lam < mu)) < 1e-10
    assert abs(res.energy - np.sum(lam[lam < mu])) < 1e-10


def test_block_diagonal_is_exact():
    s = make_lattice_system(12, 5, r_c=0.01, ell=1.5, seed=77)  # no pair within 0.01 A
    assert s.nnzb == 12
    bs, cp, ri, v = _filtered(s)
    res = O.density_submatrix(bs, cp, ri, v, 0.05)
    h = O.to_dense(bs, cp, ri, v)
    assert np.max(np.abs(O.to_dense(bs, cp, ri, res.values) - O.dense_density(h, 0.05))) < 1e-13
    assert np.all(res.dims == 5)


def test_submatrix_projector_idempotent_integer_trace():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    for j in [0, 7, 31]:
        t, rows, local = O.gather_submatrix(bs, cp, ri, v, j, mu=0.0)
        sgn, lam = O.sign_eig(t)
        p = 0.5 * (np.eye(t.shape[0]) - sgn)
        assert np.max(np.abs(p @ p - p)) < 1e-13
        assert abs(np.trace(p) - np.count_nonzero(lam < 0)) < 1e-12


def _brute_force_density(h_dense, block_size, col_ptr, row_idx, mu):
    """Independent restatement: dense indexing + Newton sign iteration, scalar loops."""
    starts = np.concatenate([[0], np.cumsum(block_size)])
    n = h_dense.shape[0]
    d = np.zeros((n, n))
    for j in range(len(block_size)):
        blocks = [int(r) for r in row_idx[col_ptr[j]:col_ptr[j + 1]]]
        idx = [p for r in blocks for p in range(starts[r], starts[r + 1])]
        m = len(idx)
        t = np.zeros((m, m))
        for a in range(m):
            for c in range(m):
                t[a, c] = h_dense[idx[a], idx[c]]
            t[a, a] -= mu
        sgn = O.sign_newton(t)
        for a in range(m):
            for q in range(starts[j], starts[j + 1]):
                cq = idx.index(q)
                d[idx[a], q] = 0.5 * ((1.0 if a == cq else 0.0) - sgn[a, cq])
    return d


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_tiny_systems(seed):
    rng = np.random.default_rng(seed)
    n_mol, b = 4, 2
    # random symmetric pattern with the diagonal, values decaying off the diagonal
    present = np.triu(rng.random((n_mol, n_mol)) < 0.6, 1)
    present = present | present.T | np.eye(n_mol, dtype=bool)
    blocks = {}
    for i in range(n_mol):
        g = rng.normal(size=(b, b))
        blocks[(i, i)] = 0.5 * (g + g.T) + np.diag([-0.8, 0.8])
        for j in range(i + 1, n_mol):
            if present[i, j]:
                blocks[(i, j)] = 0.2 * rng.normal(size=(b, b))
                blocks[(j, i)] = blocks[(i, j)].T
    col_ptr = [0]
    row_idx = []
    vals = []
    for j in range(n_mol):
        for i in range(n_mol):
            if present[i, j]:
                row_idx.append(i)
                vals.append(blocks[(i, j)].T.reshape(-1))
        col_ptr.append(len(row_idx))
    bs = np.full(n_mol, b, dtype=np.int32)
    cp, ri, v = np.array(col_ptr, dtype=np.int64), np.array(row_idx, dtype=np.int32), np.concatenate(vals)
    h = O.to_dense(bs, cp, ri, v)
    for mu in [0.0, 0.2]:
        res = O.density_submatrix(bs, cp, ri, v, mu)
        ref = _brute_force_density(h, bs, cp, ri, mu)
        got = O.to_dense(bs, cp, ri, res.values)
        assert np.max(np.abs(got - ref)) < 1e-12
        assert abs(res.trace - np.trace(ref)) < 1e-12
        assert abs(res.energy - np.sum(ref * h)) < 1e-12


def test_trace_energy_from_dense_bookkeeping():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    res = O.density_submatrix(bs, cp, ri, v, 0.1)
    d = O.to_dense(bs, cp, ri, res.values)
    h = O.to_dense(bs, cp, ri, v)
    assert abs(res.trace - np.trace(d)) < 1e-12
    assert abs(res.energy - np.trace(d @ h)) < 1e-10
    # D has exactly the pattern of H
    assert np.all(d[h == 0.0] == 0.0)


def test_global_gershgorin_hand_values_and_dense_agreement():
    # hand matrix (dense rows written out from the blocks above):
    #   row 0: [1, .5, .3, 1e-4, 0]   -> 1 -/+ 0.8001
    #   row 1: [.5, -1, -.4, 0, 1e-4] -> -1 -/+ 0.9001
    #   row 2: [.3, -.4, .2, 0, 0]    -> 0.2 -/+ 0.7
    #   rows 3, 4: one 1e-4 each      -> 0 -/+ 1e-4
    bs, cp, ri, v, _ = _hand_matrix()
    lo, hi = O.global_gershgorin(bs, cp, ri, v)
    assert abs(lo - (-1.9001)) < 1e-15 and abs(hi - 1.8001) < 1e-15
    # the bracket of the bisection equals the dense Gershgorin interval (itself pinned by hand
    # values) on the filtered water32 and on a ragged-block system
    for s in [make_workload("water32"), make_lattice_system(12, 4, 5.0, 1.5, 7)]:
        bs, cp, ri, v = _filtered(s, 1e-3)
        assert O.global_gershgorin(bs, cp, ri, v) == pytest.approx(
            O.gershgorin_bounds(O.to_dense(bs, cp, ri, v)), abs=1e-13)


def test_trace_nondecreasing_in_mu_and_bisection():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    mus = np.linspace(-1.0, 1.0, 21)
    traces = [O.density_submatrix(bs, cp, ri, v, m).trace for m in mus]
    assert np.all(np.diff(traces) >= -1e-10)
    lo, hi = O.global_gershgorin(bs, cp, ri, v)
    assert O.density_submatrix(bs, cp, ri, v, lo).trace < 1e-9
    assert O.density_submatrix(bs, cp, ri, v, hi).trace > s.n - 1e-9
    mu, res, hist = O.bisect_mu(bs, cp, ri, v, n_e=96.0, max_steps=40, tol=1e-3)
    assert abs(res.trace - 96.0) <= 1e-3 and res.mu == mu == hist[-1][0]
    # an unreachable tolerance runs all steps and the bracket keeps n_e inside
    mu, res, hist = O.bisect_mu(bs, cp, ri, v, n_e=90.5, max_steps=12, tol=0.0)
    assert len(hist) == 12
    below = [m for m, t in hist if t < 90.5]
    above = [m for m, t in hist if t >= 90.5]
    assert max(below) < min(above)


def test_symmetrize_option():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    res = O.density_submatrix(bs, cp, ri, v, 0.0)
    res_s = O.density_submatrix(bs, cp, ri, v, 0.0, symmetrize=True)
    d = O.to_dense(bs, cp, ri, res.values)
    ds = O.to_dense(bs, cp, ri, res_s.values)
    assert np.max(np.abs(ds - 0.5 * (d + d.T))) < 1e-15
    assert np.max(np.abs(d - d.T)) > 1e-6  # the unsymmetrised D is not symmetric


def test_column_subset_matches_full_run():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    full = O.density_submatrix(bs, cp, ri, v, 0.0)
    part = O.density_submatrix(bs, cp, ri, v, 0.0, columns=[3, 10])
    off = O.block_value_offsets(bs, cp, ri)
    for j in [3, 10]:
        sl = slice(off[cp[j]], off[cp[j + 1]])
        assert np.array_equal(part.values[sl], full.values[sl])
    assert np.all(part.values[off[cp[0]]:off[cp[1]]] == 0.0)


def test_threaded_equals_serial():
    s = make_workload("water32")
    bs, cp, ri, v = _filtered(s)
    a = O.density_submatrix(bs, cp, ri, v, 0.0, workers=1)
    b = O.density_submatrix(bs, cp, ri, v, 0.0, workers=4)
    assert np.array_equal(a.values, b.values)


def test_planted_mistakes_are_caught(monkeypatch):
    """Plausible mistakes planted in the oracle make a pin fail.

    References are computed with the unmodified oracle first; each mistake is
    then planted and must move the result far outside the pins' tolerances.
    """
    import oracle.submatrix as S

    sysm = make_lattice_system(5, 3, r_c=6.0, ell=1.5, seed=9)
    bs, cp, ri, v = sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values
    h = O.to_dense(bs, cp, ri, v)
    mu = 0.5  # inside the virtual band, so that D depends on the shift
    ref = _brute_force_density(h, bs, cp, ri, mu)

    def err():
        res = S.density_submatrix(bs, cp, ri, v, mu)
        off = O.block_value_offsets(bs, cp, ri)
        d = np.zeros_like(h)
        st = np.concatenate([[0], np.cumsum(bs)])
        for j in range(len(bs)):  # dense D without the (possibly patched) block reader
            for k in range(cp[j], cp[j + 1]):
                r = ri[k]
                d[st[r]:st[r + 1], st[j]:st[j + 1]] = res.values[off[k]:off[k + 1]].reshape(bs[j], bs[r]).T
        return np.max(np.abs(d - ref))

    assert err() < 1e-12
    good_block, good_sign, good_gather = S._block, S.sign_eig, S.gather_submatrix
    # 1. blocks read row-major instead of column-major (a transposed operand)
    monkeypatch.setattr(S, "_block", lambda values, off, k, br, bc: values[off[k]:off[k + 1]].reshape(br, bc))
    assert err() > 1e-3
    monkeypatch.setattr(S, "_block", good_block)
    # 2. wrong sign of the sign function (D = (I + sign)/2)
    monkeypatch.setattr(S, "sign_eig", lambda a: tuple([-good_sign(a)[0], good_sign(a)[1]]))
    assert err() > 1e-1
    monkeypatch.setattr(S, "sign_eig", good_sign)
    # 3. dropped shift (-mu I missing)
    monkeypatch.setattr(S, "gather_submatrix", lambda *a, **k: good_gather(*a[:5], 0.0, *a[6:], **k))
    assert err() > 1e-3
    monkeypatch.setattr(S, "gather_submatrix", good_gather)
    assert err() < 1e-12
