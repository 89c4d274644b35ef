"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds input generators only: point clouds, right-hand sides and the
parameter sets of the five workloads.  It contains none of the method's
arithmetic, so both the CUDA path and the CPU oracle may consume its arrays
without sharing code.
"""
from .generators import (  # noqa: F401
    WORKLOADS,
    Workload,
    make_points,
    make_rhs,
    workload,
    uniform_cube,
    gaussian_mixture,
    labeled_gaussian_mixture,
    tanh_manifold,
    batched_problems,
)
