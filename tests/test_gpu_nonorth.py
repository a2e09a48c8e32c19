"""GPU parity of the non-orthogonal form (Eq. 14 with an overlap S != I, FP64) against
oracle/nonorth.py: P = 1/2 (I - sign(S^-1 H - mu I)) S^-1 by the submatrix method at a fixed
mu, with filtering, with ragged block sizes, under the mu bisection on tr(P S), at 1024
molecules on sampled columns, and the error paths.  Tolerance: the FP64 form's 1e-10
max-abs (trace and energy 1e-10 relative)."""

import numpy as np
import pytest

import oracle as O
from synth import make_mixed_block_system, make_nonorth_pair
from tests.helpers import column_slices

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(h, s_vals, eps=0.0):
    from paper_2205_14741_gb300 import SubmatrixDensity

    c = SubmatrixDensity.from_system(h)
    c.set_precision("fp64")
    c.set_filter_threshold(eps)
    c.set_overlap(s_vals)
    return c


def _oracle(h, s_vals, eps, mu, columns=None):
    """Oracle on the filtered pattern of H (S taken on it), returned in the input layout."""
    cp, ri, hv, keep = O.filter_blocks(h.block_size, h.col_ptr, h.row_idx, h.values, eps)
    sv = O.take_blocks(h.block_size, h.col_ptr, h.row_idx, s_vals, keep)
    res = O.density_nonorth_submatrix(h.block_size, cp, ri, hv, sv, mu, columns=columns)
    off_in = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
    off_f = O.block_value_offsets(h.block_size, cp, ri)
    p_in = np.zeros(h.values.shape[0])
    kf = 0
    for k in range(h.row_idx.shape[0]):
        if keep[k]:
            p_in[off_in[k]:off_in[k + 1]] = res.values[off_f[kf]:off_f[kf + 1]]
            kf += 1
    return p_in, res, keep, (cp, ri, hv, sv)


def _check(p, tr, en, p_or, res):
    assert np.max(np.abs(p - p_or)) <= TOL
    assert abs(tr - res.trace) <= TOL * max(1.0, abs(res.trace))
    assert abs(en - res.energy) <= TOL * max(1.0, abs(res.energy))


@pytest.mark.parametrize("mu", [-0.1, 0.0, 0.15])
def test_fixed_mu_matches_oracle(mu):
    h, s = make_nonorth_pair(64, 6, 5.0, 1.5, 11)
    with _ctx(h, s.values) as c:
        c.set_mu(mu)
        c.build_density()
        p = c.get_density()
        tr, en, _ = c.get_trace()
        st = c.get_stats()
    p_or, res, _, _ = _oracle(h, s.values, 0.0, mu)
    _check(p, tr, en, p_or, res)
    assert st["n_noconv"] == 0


def test_filtered_pattern_matches_oracle():
    h, s = make_nonorth_pair(64, 6, 6.0, 1.5, 12)
    eps = 2e-2
    with _ctx(h, s.values, eps) as c:
        c.set_mu(0.0)
        c.build_density()
        p = c.get_density()
        tr, en, _ = c.get_trace()
        cp, ri = c.get_pattern()
    p_or, res, keep, (cp_or, ri_or, _, _) = _oracle(h, s.values, eps, 0.0)
    assert 0 < keep.sum() < keep.size
    assert np.array_equal(cp, cp_or) and np.array_equal(ri, ri_or)
    _check(p, tr, en, p_or, res)


def test_ragged_block_sizes():
    sizes = np.random.default_rng(5).choice([1, 3, 5, 9, 13], size=40)
    h = make_mixed_block_system(sizes, 5.0, 1.5, 13)
    # an overlap on H's pattern: identity diagonal blocks, 0.3 x H's off-diagonal blocks
    off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
    s_vals = 0.3 * h.values
    for j in range(h.n_blocks):
        for k in range(h.col_ptr[j], h.col_ptr[j + 1]):
            if h.row_idx[k] == j:
                s_vals[off[k]:off[k + 1]] = np.eye(sizes[j]).reshape(-1)
    with _ctx(h, s_vals) as c:
        c.set_mu(0.02)
        c.build_density()
        p = c.get_density()
        tr, en, _ = c.get_trace()
    p_or, res, _, _ = _oracle(h, s_vals, 0.0, 0.02)
    _check(p, tr, en, p_or, res)


def test_bisection_matches_oracle():
    h, s = make_nonorth_pair(96, 6, 5.5, 1.5, 14)
    n_e = float(h.n // 2)
    with _ctx(h, s.values) as c:
        c.set_electron_count(n_e, max_steps=40, tol=1e-2)
        c.solve_mu()
        tr, en, mu = c.get_trace()
        p = c.get_density()
        steps = c.get_stats()["bisection_steps"]
    mu_or, res_or, hist = O.bisect_mu_nonorth(h.block_size, h.col_ptr, h.row_idx, h.values, s.values, n_e, 40, 1e-2)
    # the two brackets differ in rounding only (L_j from the coupled iteration against an
    # eigendecomposition), so the midpoints agree to far below the steps of the trace
    assert abs(mu - mu_or) <= 1e-12 and steps == len(hist)
    assert abs(tr - n_e) <= 1e-2
    p_or, res, _, _ = _oracle(h, s.values, 0.0, mu)
    _check(p, tr, en, p_or, res)


def test_identity_overlap_equals_the_orthogonal_form_and_switching_back():
    h, _ = make_nonorth_pair(48, 6, 5.0, 1.5, 15)
    off = O.block_value_offsets(h.block_size, h.col_ptr, h.row_idx)
    eye = np.zeros_like(h.values)
    for j in range(h.n_blocks):
        for k in range(h.col_ptr[j], h.col_ptr[j + 1]):
            if h.row_idx[k] == j:
                eye[off[k]:off[k + 1]] = np.eye(6).reshape(-1)
    with _ctx(h, eye) as c:
        c.set_mu(0.05)
        c.build_density()
        p = c.get_density()
        tr_p = c.get_trace()[0]
        c.set_overlap(None)  # back to S = I through the orthogonal path
        c.build_density()
        d = c.get_density()
        tr_d = c.get_trace()[0]
    with _ctx(h, None) as f:
        f.set_mu(0.05)
        f.build_density()
        assert np.array_equal(f.get_density(), d)
    assert np.max(np.abs(p - d)) <= TOL and abs(tr_p - tr_d) <= TOL * abs(tr_d)


def test_sampled_columns_1024_molecules():
    h, s = make_nonorth_pair(1024, 6, 6.0, 1.5, 16)
    eps = 1e-5
    with _ctx(h, s.values, eps) as c:
        c.set_electron_count(3072.0, max_steps=40, tol=1e-2)
        c.solve_mu()
        tr, _, mu = c.get_trace()
        p = c.get_density()
        dims, iters, _ = c.get_submatrix_info()
    assert abs(tr - 3072.0) <= 1e-2
    order = np.argsort(dims)
    rng = np.random.default_rng(0)
    cols = sorted(set(order[:2].tolist()) | set(order[-3:].tolist()) | set(rng.choice(1024, 7, replace=False).tolist()))
    p_or, _, keep, _ = _oracle(h, s.values, eps, mu, columns=cols)
    err = max(float(np.max(np.abs(p[sl] - p_or[sl]))) for sl in column_slices(h, cols))
    assert err <= TOL
    assert iters.max() < 40


def test_errors():
    from paper_2205_14741_gb300 import SmxError, _lib

    h, s = make_nonorth_pair(32, 6, 5.0, 1.5, 17)
    with _ctx(h, s.values) as c:
        c.set_mu(0.0)
        c.set_precision("fp16x3")
        with pytest.raises(SmxError) as ei:
            c.build_density()
        assert ei.value.status == _lib.ERR_UNSUPPORTED
        c.set_precision("fp64")
        c.set_function("inv_sqrt")
        with pytest.raises(SmxError) as ei:
            c.build_density()
        assert ei.value.status == _lib.ERR_UNSUPPORTED
        c.set_function("density")
        c.set_staging_limit(1 << 20)  # several staging chunks: L_j and M_j cannot stay resident
        with pytest.raises(SmxError) as ei:
            c.build_density()
        assert ei.value.status == _lib.ERR_UNSUPPORTED
        c.set_staging_limit(1 << 30)
        c.build_density()  # usable again
        bad = s.values.copy()
        bad[5] = np.inf
        with pytest.raises(SmxError) as ei:
            c.set_overlap(bad)
        assert ei.value.status == _lib.ERR_NONFINITE
    # an "overlap" that is not positive definite: H itself (eigenvalues of both signs)
    with _ctx(h, h.values) as c:
        c.set_mu(0.0)
        with pytest.raises(SmxError) as ei:
            c.build_density()
            c.get_trace()
        assert ei.value.status in (_lib.ERR_NOCONV, _lib.ERR_NONFINITE)


def test_bracket_is_the_pencils_and_not_offered_to_shards():
    from paper_2205_14741_gb300 import SmxError, _lib

    h, s = make_nonorth_pair(48, 6, 5.0, 1.5, 18)
    lo_or, hi_or = O.nonorth_bracket(h.block_size, h.col_ptr, h.row_idx, h.values, s.values)
    with _ctx(h, s.values) as c:
        lo, hi = c.get_gershgorin_interval()
        # L_j from the coupled iteration against the oracle's eigendecomposition: rounding only
        assert abs(lo - lo_or) <= 1e-12 * abs(lo_or) and abs(hi - hi_or) <= 1e-12 * abs(hi_or)
        c.set_column_range(0, 24)
        with pytest.raises(SmxError) as ei:
            c.get_gershgorin_interval()
        assert ei.value.status == _lib.ERR_UNSUPPORTED
