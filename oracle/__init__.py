"""CPU oracle for the CGD-EnKF analysis step: TEST INFRASTRUCTURE, not a product path.

Plain, slow, obviously correct FP64 numpy implementations of what the GPU library
computes, each written from the paper (Lee, Liu, Valyou, Zikatanov, "A Conjugate Gradient
Formulation of the EnKF Algorithm"), with the section / equation / algorithm it follows
cited in its docstring. Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package. The GPU library neither imports nor links it,
and shares no code with it; the only code both sides use is the input generators in
`synth`, which hold none of the analysis arithmetic.

Pins (tests/test_oracle_*.py) tie every function here to something other than itself:
explicit Gauss-Jordan inverses on tiny inputs, the Kalman-filter closed form, Lemma 1,
Prop. 1, the single-observation scalar case, brute force, and Philox known-answer vectors.
"""
from .philox import philox4x32_10, uniform53_pair, obs_perturbations
from .enkf import (
    apply_H, ensemble_stats, innovations, enkf_alg1, enkf_alg2, enkf_exact, cgd_enkf,
    cgd_enkf_reduced, senkf_alg3, kalman_analysis, rel_frobenius, S_matvec, R_apply, R_dense,
    tridiag_cholesky, L_solve, L_apply,
)

__all__ = [
    "philox4x32_10", "uniform53_pair", "obs_perturbations", "apply_H", "ensemble_stats",
    "innovations", "enkf_alg1", "enkf_alg2", "enkf_exact", "cgd_enkf", "cgd_enkf_reduced",
    "senkf_alg3", "kalman_analysis", "rel_frobenius", "S_matvec", "R_apply", "R_dense",
    "tridiag_cholesky", "L_solve", "L_apply",
]
