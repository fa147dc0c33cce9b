"""Seeded synthetic least-squares workloads.

This package only draws random numbers and lays them out as a CSR matrix,
right-hand sides and column partitions.  It holds none of the solver's
arithmetic, so both the FP64 oracle and the CUDA path can take their inputs
from it without sharing any part of the method.
"""
from .grid import (  # noqa: F401
    GridLS,
    make_grid_ls,
    strip_partition,
    block_partition,
    bisection_partition,
    config_tiny,
    config_scale,
    config_precision,
    config_diff,
    config_batch_sizes,
    config_batch,
    BatchLS,
    paper_example,
    csr_from_dense,
)
