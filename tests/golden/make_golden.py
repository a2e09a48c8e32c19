"""Writes the stored oracle values under tests/golden/ (run from the repository root:
``python tests/golden/make_golden.py``).

Only the oracle (oracle/) and the seeded input generator (synth/) are used: the
stored values are the oracle's, never the CUDA path's.
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from synth import make_workload  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "water32_oracle.txt")


def main():
    s = make_workload("water32")
    res = O.density_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.0)
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(s.values.shape[0], 24, replace=False))
    mu, bres, hist = O.bisect_mu(s.block_size, s.col_ptr, s.row_idx, s.values, 96.0, max_steps=30, tol=0.5)
    lines = [
        "# Oracle values for the 32-molecule water-like system (32 x 6 blocks, cutoff 5 A, decay 1.5 A,",
        "# no filter), written by tests/golden/make_golden.py from oracle/ only: the submatrix method of",
        "# Fig. 2 with the sign of Eq. 13 by eigendecomposition and Eq. 14 with S = I.",
        "# mu = 0: trace(D), trace(D H), and D at 24 seeded positions of the input value layout.",
        f"trace {res.trace!r}",
        f"energy {res.energy!r}",
    ]
    lines += [f"d {int(k)} {float(res.values[k])!r}" for k in idx]
    lines += [
        "# bisection on trace(D) = 96 in the Gershgorin bracket (tol 0.5, at most 30 steps):",
        f"bisect_mu {mu!r}",
        f"bisect_trace {bres.trace!r}",
        f"bisect_steps {len(hist)}",
    ]
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
