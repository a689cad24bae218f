"""Seeded synthetic inputs for the EnKF analysis step.

This package is shared by the CUDA path's tests and benchmark and by the CPU oracle. It
only *draws inputs*: forecast ensembles, observation operators, observation-error
variances, truths and observations. It holds none of the analysis arithmetic (no means,
anomalies, innovations, covariances, solves or updates); the two implementations of the
analysis live elsewhere and share nothing but what this package returns.

Random numbers that the analysis itself draws (the observation perturbations E) are not
made here: both implementations draw them from their own Philox4x32-10 generator, or the
caller passes E in explicitly.
"""
from .grf import grf_fields, periodic_sqexp_eigenvalues
from .l96 import l96_tendency, l96_rk4
from .problems import (
    Problem,
    subsample_operator,
    identity_operator,
    every_kth_operator,
    obs_variances,
    grf_problem,
    workload,
    batched_problem_specs,
    batched_problems,
    L96Cycle,
    WORKLOADS,
    l96_tridiag_problem,
    ex1b_problem,
)

__all__ = [
    "grf_fields", "periodic_sqexp_eigenvalues", "l96_tendency", "l96_rk4", "Problem",
    "subsample_operator", "identity_operator", "every_kth_operator", "obs_variances",
    "grf_problem", "workload", "batched_problem_specs", "batched_problems", "L96Cycle",
    "WORKLOADS", "l96_tridiag_problem", "ex1b_problem",
]
