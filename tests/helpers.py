"""Shared test helpers: oracle evaluation in the library's output layout."""

from __future__ import annotations

import os

import numpy as np

import oracle as O


def workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def oracle_in_input_layout(sysm, eps: float, mu: float, columns=None, symmetrize=False):
    """Runs the oracle on ``sysm`` filtered with ``eps`` at ``mu``.

    Returns (D in the input pattern's value layout, oracle result, keep mask).
    Blocks dropped by the filter are zero, as in the library's output.
    """
    cp, ri, v, keep = O.filter_blocks(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, eps)
    res = O.density_submatrix(sysm.block_size, cp, ri, v, mu, workers=workers(), columns=columns,
                              symmetrize=symmetrize)
    off_in = O.block_value_offsets(sysm.block_size, sysm.col_ptr, sysm.row_idx)
    off_f = O.block_value_offsets(sysm.block_size, cp, ri)
    d_in = np.zeros(sysm.values.shape[0])
    kf = 0
    for k in range(sysm.row_idx.shape[0]):
        if keep[k]:
            d_in[off_in[k]:off_in[k + 1]] = res.values[off_f[kf]:off_f[kf + 1]]
            kf += 1
    return d_in, res, keep


def column_slices(sysm, columns):
    """Value-array slices of the given block columns (input layout)."""
    off = O.block_value_offsets(sysm.block_size, sysm.col_ptr, sysm.row_idx)
    return [slice(int(off[sysm.col_ptr[j]]), int(off[sysm.col_ptr[j + 1]])) for j in columns]


def max_abs_on_columns(a, b, sysm, columns):
    return max(float(np.max(np.abs(a[s] - b[s]))) for s in column_slices(sysm, columns))


def sample_columns(dims, k: int, seed: int = 0):
    """k block columns: the largest and smallest submatrices plus a seeded random sample."""
    dims = np.asarray(dims)
    order = np.argsort(dims)
    rng = np.random.default_rng(seed)
    pick = set(order[:2].tolist()) | set(order[-4:].tolist())
    rest = rng.choice(dims.shape[0], size=min(k, dims.shape[0]), replace=False).tolist()
    for j in rest:
        if len(pick) >= k:
            break
        pick.add(j)
    return sorted(pick)
