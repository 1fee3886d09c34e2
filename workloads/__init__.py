"""Seeded synthetic inputs for the RSM hot path.

This package holds input generators only: it builds Y (values) and W (the
known-entry mask) with the shapes and distributions of the paper's workloads
and of the five benchmark configurations. It contains none of the method's
arithmetic (no column sampling, no row selection, no SVD, no accumulation),
so both the FP64 oracle and the CUDA path may use it.
"""
from .synthetic import (  # noqa: F401
    Problem,
    lowrank_problem,
    trajectory_problem,
    batched_problem_specs,
    batched_problem,
    LARGE_SERVING,
    serving_arrivals,
    config_problem,
    CONFIGS,
)
