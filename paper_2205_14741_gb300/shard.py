"""Sharding the submatrix method over several GPUs (host logic).

The submatrices are independent (Fig. 2: one dense sign function per block
column), so a multi-GPU run gives each rank a contiguous range of block
columns; the only exchange is the 16-byte sum of (trace(D), trace(DH)) over
the ranks at every bisection step for mu (Eq. 14).  Each rank's context is
restricted with ``set_column_range``; every build runs in the CUDA library,
this module only partitions and drives the bisection.
"""

from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def partition_columns(dims: Sequence[int], world: int) -> list[tuple[int, int]]:
    """Contiguous block-column ranges, one per rank, balanced by the Newton-Schulz work sum n_j^3.

    Range r ends at the first column whose prefix work reaches (r + 1)/world of
    the total; every range is non-empty (world <= number of columns).
    """
    n = len(dims)
    if world < 1 or world > n:
        raise ValueError(f"cannot split {n} block columns over {world} ranks")
    w = np.asarray(dims, dtype=np.float64) ** 3
    prefix = np.cumsum(w)
    total = prefix[-1]
    bounds = [0]
    for r in range(1, world):
        cut = int(np.searchsorted(prefix, total * r / world, side="left")) + 1
        cut = max(cut, bounds[-1] + 1)           # non-empty
        cut = min(cut, n - (world - r))          # leave one column per remaining rank
        bounds.append(cut)
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def solve_mu_sharded(ctx, n_e: float, allreduce_sum: Callable[[np.ndarray], np.ndarray],
                     max_steps: int = 30, tol: float = 1e-2):
    """Bisection for mu over sharded contexts (the same rule as ``smx_solve_mu``).

    ``ctx`` is this rank's context (restricted to its block columns) and
    ``allreduce_sum`` returns the elementwise sum over the ranks of a float64
    array of 2 (trace(D), trace(DH)).  Every rank takes the same decisions, so
    all end on the same mu.  Returns (mu, trace, energy, builds).
    """
    lo, hi = ctx.get_gershgorin_interval()
    mid, tr, en, steps = 0.5 * (lo + hi), 0.0, 0.0, 0
    for steps in range(1, max_steps + 1):
        mid = 0.5 * (lo + hi)
        ctx.set_mu(mid)
        ctx.build_density()
        t, e, _ = ctx.get_trace()
        tr, en = (float(x) for x in allreduce_sum(np.array([t, e], dtype=np.float64)))
        if abs(tr - n_e) <= tol:
            break
        if tr < n_e:
            lo = mid
        else:
            hi = mid
    return mid, tr, en, steps
