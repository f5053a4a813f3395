"""Seeded synthetic inputs for the shifted-Hessenberg eigenvector solve.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic: it only draws
random numbers (a counter-based SplitMix64 generator), builds test matrices
with known eigenvalues, reduces them to Hessenberg form with LAPACK (the
precursor step of the method, not the method) and picks shifts and starting
vectors.

The matrices follow the paper's first test problem (Sec. 5.2: known,
well-separated eigenvalues on a (quasi-)triangular T, then an orthogonal
similarity and a Hessenberg reduction) with the sizes and distributions of
the five workload configurations, plus the paper's second test problem
(the "bad" H2 and "good" H3 systems, Sec. 5.2), companion matrices and
graded matrices D H D^-1.
"""
from .rng import splitmix64, uniform, normal
from .matrices import (
    haar_orthogonal,
    quasi_triangular,
    hessenberg_reduce,
    paper_h2,
    paper_h3,
    paper_r2_q2,
    companion,
    graded,
    unit_columns,
)
from .configs import (
    Instance,
    config0,
    config1,
    config2,
    config3,
    config3_sizes,
    batch_instance,
    serving_pool,
    serving_requests,
    SERVE_SIZES,
    small_instance,
    column_offsets,
)

__all__ = [
    "splitmix64", "uniform", "normal", "haar_orthogonal", "quasi_triangular",
    "hessenberg_reduce", "paper_h2", "paper_h3", "paper_r2_q2", "companion", "graded",
    "unit_columns", "Instance", "config0", "config1", "config2", "config3", "config3_sizes",
    "batch_instance", "serving_pool", "serving_requests", "SERVE_SIZES", "small_instance",
    "column_offsets",
]
