"""Host emulation of the low-precision bulk phase (Section 3's FP16 products with FP32
accumulation), to document which formats can reach the 1e-5 bound on D at all: the Newton-Schulz
sign iteration on one water-like submatrix with every product's operands rounded to a 16-bit or
8-bit format (FP8 e4m3 with a per-matrix scale, as the tensor cores would take them) and FP32
accumulation, against the oracle's eigendecomposition.  No GPU: numpy rounding and float32
matrix products.  The split FP16 form (hi + lo, three products) reaches the bound; single-pass
FP16 and BF16 stall near 6e-4 and 6e-3 on this 114 x 114 submatrix; FP8 near 4e-2, so no FP8 form is built.
"""

import numpy as np
import pytest

import oracle as O
from synth import make_workload


def round_fp16(x):
    return x.astype(np.float16).astype(np.float32)


def round_bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    r = ((b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).view(np.float32)
    return r


def round_e4m3(x):
    """FP8 e4m3 (4 significant bits, normal range down to 2^-6, subnormal grid 2^-9, max 448)
    after scaling the matrix so that its largest entry maps to 448."""
    x = np.asarray(x, dtype=np.float64)
    amax = float(np.max(np.abs(x)))
    if amax == 0.0:
        return x.astype(np.float32)
    s = 448.0 / amax
    y = x * s
    m, e = np.frexp(y)  # y = m 2^e, |m| in [0.5, 1)
    e = np.maximum(e, -5)  # below 2^-6 the subnormal grid 2^-9 applies
    q = np.round(y / 2.0 ** (e - 4)) * 2.0 ** (e - 4)
    q = np.clip(q, -448.0, 448.0)
    return (q / s).astype(np.float32)


def split_fp16(x):
    hi = round_fp16(x)
    return hi, round_fp16(x.astype(np.float32) - hi)


def product(a, b, fmt):
    a = a.astype(np.float32)
    b = b.astype(np.float32)
    if fmt == "fp16x3":
        ah, al = split_fp16(a)
        bh, bl = split_fp16(b)
        return ah @ bh + (ah @ bl + al @ bh)
    r = {"fp16": round_fp16, "bf16": round_bf16, "e4m3": round_e4m3}[fmt]
    return r(a) @ r(b)


def ns_density(a, fmt, tau, max_iter=60):
    lo, hi = O.gershgorin_bounds(a)
    x = (a / max(abs(lo), abs(hi))).astype(np.float32)
    n = a.shape[0]
    eye = np.eye(n, dtype=np.float32)
    for _ in range(max_iter):
        z = product(x, x, fmt)
        r = float(np.linalg.norm(z - eye))
        x = product(x, 1.5 * eye - 0.5 * z, fmt)
        if r <= tau:
            break
    return 0.5 * (np.eye(n) - x.astype(np.float64))


@pytest.fixture(scope="module")
def submatrix():
    s = make_workload("water32")
    a, rows, local = O.gather_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 5, 0.0)
    d = O.dense_density(a, 0.0)
    return a, d


@pytest.mark.parametrize("fmt,tau,lo,hi", [
    ("fp16x3", 2e-3, 0.0, 1e-5),
    ("fp16", 5e-2, 1e-5, 5e-3),
    ("bf16", 5e-2, 1e-4, 5e-2),
    ("e4m3", 5e-1, 1e-2, 1.0),
])
def test_error_of_each_bulk_format(submatrix, fmt, tau, lo, hi):
    a, d = submatrix
    err = float(np.max(np.abs(ns_density(a, fmt, tau) - d)))
    assert lo <= err <= hi, f"{fmt}: max|D - oracle| = {err:.2e}"


def test_e4m3_rounding_is_the_format():
    # 4 significant bits: 1, 1.125, ..., 1.875 are exact, 1.0625 rounds to even
    x = np.array([448.0, 1.0, 1.125, 1.875, 1.0625, 0.0], dtype=np.float64)
    q = round_e4m3(x)
    assert q[0] == 448.0 and q[1] == 1.0 and q[2] == 1.125 and q[3] == 1.875 and q[4] in (1.0, 1.125)
    assert q[5] == 0.0
