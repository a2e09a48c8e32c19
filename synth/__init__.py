"""Seeded synthetic inputs for the submatrix density-matrix method.

This package only generates inputs (positions, block-sparse Kohn-Sham-like
matrices, test matrices with a prescribed spectrum). It contains none of the
method's arithmetic: no filtering, no sign function, no density matrix. Both
the CPU oracle's tests and the GPU harness draw their inputs from here.
"""

from .water import (  # noqa: F401
    BlockCSC,
    WORKLOADS,
    make_workload,
    make_lattice_system,
    make_mixed_block_system,
    make_overlap_system,
    make_nonorth_pair,
    make_slab_system,
    md_trajectory,
    keyed_normals,
    spectrum_matrix,
)
