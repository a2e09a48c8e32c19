"""Host restatement of the integer-pipe FP64 <-> FP32 conversions the small kernels use
(``d2f_rn`` and ``f2d`` in the device header): the same bit operations on numpy integers
against numpy's IEEE conversions (round to nearest even), including exact ties, carries into
the exponent and overflow to infinity.  Values outside the normal FP32 range take the
conversion instruction in the kernel and are only checked to be routed there."""

import numpy as np

FALLBACK = object()


def d2f_bits(x: float):
    b = int(np.float64(x).view(np.uint64))
    hi, lo = b >> 32, b & 0xFFFFFFFF
    ef = ((hi >> 20) & 0x7FF) - 896
    if not 1 <= ef <= 254:
        return FALLBACK
    r = (hi & 0x80000000) | (ef << 23) | ((hi & 0xFFFFF) << 3) | (lo >> 29)
    rem = lo & 0x1FFFFFFF
    if rem > 0x10000000 or (rem == 0x10000000 and (r & 1)):
        r += 1
    return np.uint32(r & 0xFFFFFFFF).view(np.float32)


def f2d_bits(f: np.float32):
    u = int(np.float32(f).view(np.uint32))
    e = (u >> 23) & 0xFF
    if e in (0, 0xFF):
        return FALLBACK
    hi = (u & 0x80000000) | ((e + 896) << 20) | ((u & 0x7FFFFF) >> 3)
    lo = (u << 29) & 0xFFFFFFFF
    return np.uint64((hi << 32) | lo).view(np.float64)


def _check_d2f(xs):
    n = 0
    for x in xs:
        got = d2f_bits(x)
        if got is FALLBACK:
            continue
        want = np.float32(x)
        assert got.view(np.uint32) == want.view(np.uint32), (x, got, want)
        n += 1
    return n


def test_d2f_random_magnitudes():
    rng = np.random.default_rng(1)
    xs = rng.standard_normal(20000) * np.exp(rng.uniform(-80, 80, 20000))
    assert _check_d2f(xs) > 19000


def test_d2f_ties_and_carries():
    rng = np.random.default_rng(2)
    f = rng.standard_normal(4000).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    base = (f.astype(np.float64)).view(np.uint64)
    half = np.uint64(1 << 28)
    # exact ties (even and odd last kept bit), one below and one above a tie
    cases = np.concatenate([base + half, base + half - np.uint64(1), base + half + np.uint64(1),
                            base + np.uint64((1 << 29) - 1)])
    assert _check_d2f(cases.view(np.float64)) == cases.shape[0]
    # mantissa all ones: the carry moves into the exponent; at the top of the range it gives inf
    top = np.float64(np.finfo(np.float32).max) + np.float64(2.0 ** 103)  # a tie above FLT_MAX rounds to inf
    assert d2f_bits(top) == np.float32(np.inf)
    ones = np.uint64(0x3FEFFFFFFFFFFFFF).view(np.float64)  # just below 1.0
    assert d2f_bits(ones) == np.float32(1.0)
    assert u.shape[0] == 4000


def test_d2f_routes_the_rest_to_the_instruction():
    for x in [0.0, -0.0, 1e-40, -3e-39, 1e39, np.inf, -np.inf, np.nan, 5e-324]:
        assert d2f_bits(x) is FALLBACK


def test_f2d_exact():
    rng = np.random.default_rng(3)
    f = (rng.standard_normal(20000) * np.exp(rng.uniform(-80, 80, 20000))).astype(np.float32)
    n = 0
    for v in f:
        got = f2d_bits(v)
        if got is FALLBACK:
            continue
        assert got.view(np.uint64) == np.float64(v).view(np.uint64)
        n += 1
    assert n > 19000
    for v in [0.0, -0.0, 1e-45, np.inf, np.nan]:
        assert f2d_bits(np.float32(v)) is FALLBACK
