"""Pins of oracle/blockcg.py: block CG (O'Leary) against per-column CG and the exact solve,
with the closed-form termination the structure of S gives; the Prop. 1 and Prop. 3 error
bounds (Sec. 4) against a hand-evaluated spectrum and against the oracle's CG errors on the
random-vector workload of Example 1b, where Prop. 3 is the sharper one as the spectrum
clusters (Fig. 4)."""
import numpy as np
import pytest

import oracle
from oracle import blockcg as bc
import synth


def _system(m, N, seed, perturb=False, r_lo=1.0, r_hi=1.0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, N)) + rng.standard_normal(m)[:, None]
    rowptr, col, w = synth.identity_operator(m)
    r = rng.uniform(r_lo, r_hi, m)
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N)) if perturb else None
    _, _, Z, _, HA = oracle.ensemble_stats(X, rowptr, col, w)
    D = oracle.innovations(y, Z, E)
    S = HA @ HA.T / (N - 1) + np.diag(r)
    return S, D, r


def test_block_cg_with_one_column_is_cg():
    S, D, r = _system(30, 6, 1)
    d = D[:, :1]
    for k in (1, 3, 7):
        Xb, _, _ = bc.block_cg(lambda V: S @ V, d, fixed_iters=k)
        Xc, _, _, _ = oracle.enkf._cg_columns(lambda V: S @ V, d, 1e-30, 1000, fixed_iters=k)
        assert np.max(np.abs(Xb - Xc)) <= 1e-12 * np.max(np.abs(Xc))


@pytest.mark.parametrize("perturb,r_lo,r_hi,steps", [(False, 0.3, 0.3, 1), (True, 0.3, 0.3, 2),
                                                      (True, 0.5, 1.5, 2)])
def test_block_pcg_terminates_in_the_block_krylov_space_of_the_solution(perturb, r_lo, r_hi, steps):
    """S = HA HA^T/(N-1) + R: the solution R^{-1}(D - HA W) lies in span(R^{-1} D, R^{-1} HA).
    Without perturbations D = (y - zbar) 1^T - HA already spans both when R = s I (one block
    step); otherwise two block steps of CG preconditioned by R reach it."""
    S, D, r = _system(200, 10, 3, perturb, r_lo, r_hi)
    Xs = np.linalg.solve(S, D)
    Xb, k, res = bc.block_cg(lambda V: S @ V, D, fixed_iters=steps, precond=lambda R: R / r[:, None])
    assert np.linalg.norm(Xb - Xs) <= 1e-9 * np.linalg.norm(Xs)
    # per-column CG needs many more steps on the same system
    _, it, _, _ = oracle.enkf._cg_columns(lambda V: S @ V, D, 1e-10, 1000)
    assert it.max() > 3 * steps


def test_prop3_on_a_spectrum_evaluated_by_hand():
    # eigenvalues {1 (x5), 10, 20}: with the two large ones as sigma_0 (l = 2) and
    # sigma_1 = {1}: C = |1 - 1/10| |1 - 1/20| = 0.855, cond_eff = 1, so the bound is 2 C at
    # r = 2 and 0 from r = 3 on (CG ends in 3 steps on 3 distinct eigenvalues)
    eigs = np.array([1.0] * 5 + [10.0, 20.0])
    assert bc.prop3_bound(eigs, 2, 0, 2) == pytest.approx(2 * 0.9 * 0.95, rel=1e-15)
    assert bc.prop3_bound(eigs, 3, 0, 2) == 0.0
    assert bc.prop3_bound(eigs, 1, 0, 2) is None            # r < l
    # no outliers: Prop. 3 is the classical bound
    assert bc.prop3_bound(eigs, 4, 0, 0) == pytest.approx(bc.classical_bound(eigs, 4), rel=1e-15)
    k = 20.0
    assert bc.classical_bound(eigs, 2) == pytest.approx(2 * ((k ** 0.5 - 1) / (k ** 0.5 + 1)) ** 2, rel=1e-15)


@pytest.mark.parametrize("m", [20, 200, 1000])
def test_cg_errors_lie_below_both_bounds_on_example_1b(m):
    p = synth.ex1b_problem(m)
    N = p.N
    _, _, Z, _, HA = oracle.ensemble_stats(p.Xf, p.rowptr, p.col, p.w)
    D = oracle.innovations(p.y, Z, None)
    S = HA @ HA.T / (N - 1) + np.diag(p.r)
    eigs = np.linalg.eigvalsh(S)
    _, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, None, fixed_iters=40, keep_iterates=True)
    err = bc.energy_errors(S, D, info["iterates"])
    sharper = 0
    for r in range(1, 40):
        cl = bc.classical_bound(eigs, r) * err[0]
        p3 = bc.prop3_best(eigs, r, max_out=8) * err[0]
        floor = 1e-9 * err[0]              # the bounds are exact-arithmetic; CG stops at round-off
        if cl > floor:
            assert err[r] <= cl * (1 + 1e-9), (m, r)
        if p3 > floor:
            assert err[r] <= p3 * (1 + 1e-9), (m, r)
        if r == 10:
            ratio10 = p3 / cl
    # at m = 1000 the spectrum is a cluster at 1 with N - 1 outliers above 7 (Fig. 4a), and
    # Prop. 3 is far sharper than the classical bound (Fig. 4b)
    if m == 1000:
        assert ratio10 < 1e-2, ratio10
