"""The oracle against its stored values (tests/golden/water32_oracle.txt, written by
tests/golden/make_golden.py from oracle/ only): a change to the oracle's arithmetic shows
here.  The GPU path is compared with the same file in tests/test_gpu_parity.py.
"""

import os

import numpy as np

import oracle as O
from synth import make_workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "water32_oracle.txt")


def load_golden(path=GOLDEN):
    g = {"d": {}}
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        key, *rest = line.split()
        if key == "d":
            g["d"][int(rest[0])] = float(rest[1])
        else:
            g[key] = float(rest[0])
    return g


def test_oracle_reproduces_stored_values():
    g = load_golden()
    s = make_workload("water32")
    res = O.density_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.0)
    assert abs(res.trace - g["trace"]) <= 1e-12 * abs(g["trace"])
    assert abs(res.energy - g["energy"]) <= 1e-12 * abs(g["energy"])
    for k, v in g["d"].items():
        assert abs(res.values[k] - v) <= 1e-13, k
    mu, bres, hist = O.bisect_mu(s.block_size, s.col_ptr, s.row_idx, s.values, 96.0, max_steps=30, tol=0.5)
    assert abs(mu - g["bisect_mu"]) <= 1e-14 and len(hist) == int(g["bisect_steps"])
    assert abs(bres.trace - g["bisect_trace"]) <= 1e-10
    assert len(g["d"]) == 24 and np.isfinite(list(g["d"].values())).all()
