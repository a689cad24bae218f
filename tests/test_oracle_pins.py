"""Pins of the CPU oracle to things other than itself (no GPU).

Each test ties an oracle function to an independent fact: an explicit Gauss-Jordan
inverse evaluated with pure-Python loops, the Kalman-filter closed form (Sec. 2.2), the
single-observation scalar gain (Sec. 2.4), Lemma 1, Prop. 1, the Galerkin characterisation
of CG iterates, published Philox known-answer vectors, and limiting / invariance cases.
A plausible slip in the oracle (a dropped 1/(N-1), a sign, a transposed operand, a missing
E) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_problem(n, N, m, seed, r_lo=0.5, r_hi=1.5):
    rng = np.random.default_rng(seed)
    Xf = rng.standard_normal((n, N)) + rng.standard_normal(n)[:, None]
    # a general CSR operator: 1..3 weighted entries per row
    rowptr, col, w = [0], [], []
    for i in range(m):
        k = int(rng.integers(1, 4))
        col += list(rng.choice(n, size=k, replace=False))
        w += list(rng.uniform(-1.5, 1.5, size=k))
        rowptr.append(len(col))
    r = rng.uniform(r_lo, r_hi, size=m)
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N)) * np.sqrt(r)[:, None]
    return (Xf, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(w), r, y, E)


# ---------------------------------------------------------------- pure-Python brute force
def _gauss_jordan_inverse(M):
    n = len(M)
    a = [list(map(float, row)) + [1.0 if i == j else 0.0 for j in range(n)]
         for i, row in enumerate(M)]
    for c in range(n):
        piv = max(range(c, n), key=lambda i: abs(a[i][c]))
        a[c], a[piv] = a[piv], a[c]
        p = a[c][c]
        a[c] = [v / p for v in a[c]]
        for i in range(n):
            if i != c and a[i][c] != 0.0:
                f = a[i][c]
                a[i] = [vi - f * vc for vi, vc in zip(a[i], a[c])]
    return [row[n:] for row in a]


def _brute_force_enkf(Xf, rowptr, col, w, r, y, E):
    """X_a = X_f + Psi_x Psi_z^{-1} (Y + E - Z) with Psi_x, Psi_z the sample cross- and
    auto-covariances of Sec. 2.3 written as explicit sums, the inverse by Gauss-Jordan."""
    n, N = len(Xf), len(Xf[0])
    m = len(r)
    Z = [[0.0] * N for _ in range(m)]
    for i in range(m):
        for k in range(rowptr[i], rowptr[i + 1]):
            for j in range(N):
                Z[i][j] += w[k] * Xf[col[k]][j]
    xbar = [sum(Xf[a]) / N for a in range(n)]
    zbar = [sum(Z[i]) / N for i in range(m)]
    Psi_x = [[sum((Xf[a][j] - xbar[a]) * (Z[i][j] - zbar[i]) for j in range(N)) / (N - 1)
              for i in range(m)] for a in range(n)]
    Psi_z = [[sum((Z[i][j] - zbar[i]) * (Z[k][j] - zbar[k]) for j in range(N)) / (N - 1)
              + (r[i] if i == k else 0.0) for k in range(m)] for i in range(m)]
    Sinv = _gauss_jordan_inverse(Psi_z)
    K = [[sum(Psi_x[a][k] * Sinv[k][i] for k in range(m)) for i in range(m)] for a in range(n)]
    innov = [[y[i] + E[i][j] - Z[i][j] for j in range(N)] for i in range(m)]
    return [[Xf[a][j] + sum(K[a][i] * innov[i][j] for i in range(m)) for j in range(N)]
            for a in range(n)]


@pytest.mark.parametrize("n,N,m,seed", [(5, 4, 3, 0), (6, 3, 5, 1), (4, 6, 4, 2), (7, 2, 3, 3)])
def test_alg1_matches_gauss_jordan_brute_force(n, N, m, seed):
    Xf, rowptr, col, w, r, y, E = _tiny_problem(n, N, m, seed)
    ref = np.array(_brute_force_enkf(Xf.tolist(), rowptr.tolist(), col.tolist(), w.tolist(),
                                     r.tolist(), y.tolist(), E.tolist()))
    got = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # E = 0 is the paper's unperturbed (deterministic) EnKF
    ref0 = np.array(_brute_force_enkf(Xf.tolist(), rowptr.tolist(), col.tolist(), w.tolist(),
                                      r.tolist(), y.tolist(), np.zeros_like(E).tolist()))
    got0 = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, None)
    assert np.max(np.abs(got0 - ref0)) <= 1e-12 * max(1.0, np.max(np.abs(ref0)))


@pytest.mark.parametrize("n,N,m", [(30, 8, 12), (40, 20, 20), (200, 16, 150), (64, 40, 10)])
def test_alg2_woodbury_equals_alg1_dense(n, N, m):
    Xf, rowptr, col, w, r, y, E = _tiny_problem(n, N, m, n + N + m)
    a1 = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    a2 = oracle.enkf_alg2(Xf, rowptr, col, w, r, y, E)
    assert oracle.rel_frobenius(a2, a1) < 1e-11


def test_alg2_equals_alg1_on_grf_workload():
    p = synth.workload("grf512_N64_m65536", 3, scale=16)   # n=1024, m=256, N=64
    E = oracle.obs_perturbations(11, 5, p.r, p.N)
    a1 = oracle.enkf_alg1(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    a2 = oracle.enkf_alg2(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(a2, a1) < 1e-11


# ---------------------------------------------------------------- Kalman filter pins
def test_ensemble_analysis_is_kalman_gain_with_sample_covariance():
    """Sec. 2.2 with P = the sample covariance of Sec. 2.3: X_a = X_f + K (Y + E - H X_f),
    K = P H^T (H P H^T + R)^{-1}, forming the n x n P and a dense H explicitly."""
    n, N, m = 9, 12, 6
    Xf, rowptr, col, w, r, y, E = _tiny_problem(n, N, m, 42)
    Hd = np.zeros((m, n))
    for i in range(m):
        for k in range(rowptr[i], rowptr[i + 1]):
            Hd[i, col[k]] += w[k]
    mean = Xf.mean(axis=1, keepdims=True)
    Pf = (Xf - mean) @ (Xf - mean).T / (N - 1)
    _, _, K = oracle.kalman_analysis(mean[:, 0], Pf, Hd, np.diag(r), y)
    ref = Xf + K @ (y[:, None] + E - Hd @ Xf)
    for fn in (oracle.enkf_alg1, oracle.enkf_alg2):
        assert oracle.rel_frobenius(fn(Xf, rowptr, col, w, r, y, E), ref) < 1e-12
    Xa, _ = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-14, max_iter=200)
    assert oracle.rel_frobenius(Xa, ref) < 1e-11


def test_kalman_filter_closed_form_itself():
    """The KF helper against the scalar closed form: x_a = (r x + p y)/(p + r), P_a = p r/(p + r)."""
    xa, Pa, K = oracle.kalman_analysis(np.array([1.0]), np.array([[4.0]]), np.array([[1.0]]),
                                       np.array([[1.0]]), np.array([3.0]))
    assert abs(xa[0] - (1.0 * 1.0 + 4.0 * 3.0) / 5.0) < 1e-15
    assert abs(Pa[0, 0] - 4.0 / 5.0) < 1e-15


def test_perturbed_enkf_converges_to_kalman_filter_as_N_grows():
    """Linear-Gaussian case: prior N(mu, P), perturbed observations E ~ N(0, R). As N grows
    the analysis-ensemble mean tends to the KF mean and its covariance to (I - K H) P, with
    Monte-Carlo error ~ N^{-1/2}."""
    n, m = 3, 2
    rng = np.random.default_rng(7)
    Lp = np.array([[1.0, 0, 0], [0.5, 0.8, 0], [-0.3, 0.2, 0.6]])
    P = Lp @ Lp.T
    mu = np.array([0.5, -1.0, 2.0])
    rowptr, col, w = np.array([0, 1, 3], np.int32), np.array([0, 1, 2], np.int32), np.array([1.0, 1.0, -0.5])
    Hd = np.array([[1.0, 0, 0], [0, 1.0, -0.5]])
    r = np.array([0.4, 0.9])
    y = np.array([1.2, -0.4])
    xa_kf, Pa_kf, _ = oracle.kalman_analysis(mu, P, Hd, np.diag(r), y)
    errs_mean, errs_cov = [], []
    for N in (1000, 10000, 100000):
        Xf = mu[:, None] + Lp @ rng.standard_normal((n, N))
        E = np.sqrt(r)[:, None] * rng.standard_normal((m, N))
        Xa = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
        errs_mean.append(np.linalg.norm(Xa.mean(axis=1) - xa_kf) / np.linalg.norm(xa_kf))
        errs_cov.append(np.linalg.norm(np.cov(Xa) - Pa_kf) / np.linalg.norm(Pa_kf))
    assert errs_mean[-1] < 0.01 and errs_cov[-1] < 0.02
    assert errs_mean[-1] < errs_mean[0] and errs_cov[-1] < errs_cov[0]
    # the unperturbed form (E = 0) does not reach (I - K H) P: it shrinks the spread too far
    Xf = mu[:, None] + Lp @ rng.standard_normal((n, 100000))
    Xa0 = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, None)
    assert np.trace(np.cov(Xa0)) < 0.97 * np.trace(Pa_kf)


# ---------------------------------------------------------------- scalar / limiting cases
def test_single_observation_scalar_gain():
    """m = 1: K e_1 = psi_x / psi_z (Sec. 2.4), evaluated with explicit sums; the serial
    EnKF (Algorithm 3) is then exact as well."""
    n, N = 6, 5
    Xf, rowptr, col, w, r, y, E = _tiny_problem(n, N, 1, 9)
    z = [sum(w[k] * Xf[col[k], j] for k in range(rowptr[0], rowptr[1])) for j in range(N)]
    zb = sum(z) / N
    xb = [sum(Xf[a]) / N for a in range(n)]
    psi_x = [sum((Xf[a, j] - xb[a]) * (z[j] - zb) for j in range(N)) / (N - 1) for a in range(n)]
    psi_z = sum((z[j] - zb) ** 2 for j in range(N)) / (N - 1) + r[0]
    ref = np.array([[Xf[a, j] + psi_x[a] / psi_z * (y[0] + E[0, j] - z[j]) for j in range(N)]
                    for a in range(n)])
    for fn in (oracle.enkf_alg1, oracle.enkf_alg2, oracle.senkf_alg3):
        got = fn(Xf, rowptr, col, w, r, y, E)
        assert np.max(np.abs(got - ref)) < 1e-13


def test_huge_observation_error_leaves_forecast_unchanged():
    Xf, rowptr, col, w, r, y, E = _tiny_problem(20, 8, 10, 5)
    big = np.full_like(r, 1e14)
    for fn in (oracle.enkf_alg1, oracle.enkf_alg2):
        Xa = fn(Xf, rowptr, col, w, big, y, None)
        assert oracle.rel_frobenius(Xa, Xf) < 1e-12


def test_observation_order_does_not_matter():
    Xf, rowptr, col, w, r, y, E = _tiny_problem(30, 10, 12, 6)
    perm = np.random.default_rng(1).permutation(12)
    rp, cl, ww = [0], [], []
    for i in perm:
        cl += list(col[rowptr[i]:rowptr[i + 1]])
        ww += list(w[rowptr[i]:rowptr[i + 1]])
        rp.append(len(cl))
    a = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    b = oracle.enkf_alg1(Xf, np.array(rp, np.int32), np.array(cl, np.int32), np.array(ww),
                         r[perm], y[perm], E[perm])
    assert oracle.rel_frobenius(b, a) < 1e-13


def test_analysis_mean_unaffected_by_member_order():
    Xf, rowptr, col, w, r, y, E = _tiny_problem(15, 7, 9, 8)
    perm = np.random.default_rng(2).permutation(7)
    a = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    b = oracle.enkf_alg1(Xf[:, perm], rowptr, col, w, r, y, E[:, perm])
    assert np.max(np.abs(a[:, perm] - b)) < 1e-12


def _analyses():
    """Every exact or converged analysis form of the oracle, as functions of
    (Xf, rowptr, col, w, r, y, E)."""
    return {
        "alg1": oracle.enkf_alg1,
        "alg2": oracle.enkf_alg2,
        "cgd": lambda *a: oracle.cgd_enkf(*a, tol=1e-14, max_iter=500)[0],
        "reduced": lambda *a: oracle.cgd_enkf_reduced(*a, tol=1e-14, max_iter=500)[0],
    }


@pytest.mark.parametrize("s", [1e-6, 1e6])
def test_analysis_scales_with_the_units_of_state_and_observations(s):
    """The same problem in other units (X_f, y and E times s, R times s^2) has S, D and the
    anomalies scaled by s^2, s and s, so the analysis scales by s. Using sqrt(r) for r, or
    an unscaled perturbation, would break it."""
    Xf, rowptr, col, w, r, y, E = _tiny_problem(40, 8, 20, 11)
    for name, fn in _analyses().items():
        a = fn(Xf, rowptr, col, w, r, y, E)
        b = fn(s * Xf, rowptr, col, w, s * s * r, s * y, s * E)
        assert oracle.rel_frobenius(b / s, a) < 1e-10, name


def test_analysis_follows_a_shift_of_the_state():
    """Adding one state c to every member and H c to y leaves the anomalies and the
    innovations as they were, so every member's analysis moves by c. Forming the gain from
    the uncentred observed ensemble instead of HA would break it."""
    Xf, rowptr, col, w, r, y, E = _tiny_problem(40, 8, 20, 12)
    c = 3.0 + np.random.default_rng(5).standard_normal(40)
    Hc = oracle.apply_H(rowptr, col, w, c[:, None])[:, 0]
    for name, fn in _analyses().items():
        a = fn(Xf, rowptr, col, w, r, y, E)
        b = fn(Xf + c[:, None], rowptr, col, w, r, y + Hc, E)
        assert np.max(np.abs(b - (a + c[:, None]))) < 1e-9 * np.max(np.abs(b)), name


# ---------------------------------------------------------------- CG pins
def _krylov_galerkin_iterate(S, d, k):
    """The k-th CG iterate from 0 is the Galerkin solution on the Krylov space
    K_k(S, d): x_k = V (V^T S V)^{-1} V^T d with V an orthonormal basis of K_k."""
    V = np.empty((len(d), k))
    v = d / np.linalg.norm(d)
    for i in range(k):
        V[:, i] = v
        v = S @ v
        v -= V[:, : i + 1] @ (V[:, : i + 1].T @ v)
        v -= V[:, : i + 1] @ (V[:, : i + 1].T @ v)
        v /= np.linalg.norm(v)
    return V @ np.linalg.solve(V.T @ S @ V, V.T @ d)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_cg_iterates_are_krylov_galerkin_solutions(k):
    p = synth.workload("grf512_N64_m65536", 4, scale=32)   # n=256, m=64, N=64
    E = oracle.obs_perturbations(3, 1, p.r, p.N)
    _, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, fixed_iters=k)
    Zhat, D = info["Zhat"], info["D"]
    S = Zhat @ Zhat.T / (p.N - 1) + np.diag(p.r)
    for j in (0, 17, 63):
        ref = _krylov_galerkin_iterate(S, D[:, j], k)
        assert np.linalg.norm(info["Z"][:, j] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_lemma1_equal_variances_converge_within_N_plus_1_steps():
    """Lemma 1: with R = sigma^2 I the system matrix is sigma^2 (I + P P^T) with rank(P) < N,
    so CG reaches the solution within N+1 steps (here to relative residual 1e-12)."""
    for N, m, seed in ((8, 200, 0), (16, 400, 1), (20, 20, 2)):
        Xf, rowptr, col, w, r, y, E = _tiny_problem(3 * m, N, m, seed)
        r = np.full(m, 0.7)
        _, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-12, max_iter=N + 1)
        assert info["iters"].max() <= N + 1
        assert info["relres"].max() <= 1e-12
        # a non-uniform R is not covered by the lemma and needs more steps here
    Xf, rowptr, col, w, r, y, E = _tiny_problem(600, 8, 200, 0, r_lo=0.05, r_hi=5.0)
    _, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-12, max_iter=500)
    assert info["iters"].max() > 9


@pytest.mark.parametrize("m", [10, 20, 200])
def test_prop1_classical_cg_bound(m):
    """Example 1b / Prop. 1: R = I, H = I; the S-norm error of every CG iterate obeys
    ||e_r||_S <= 2 ((sqrt(k) - 1)/(sqrt(k) + 1))^r ||e_0||_S, k = cond(S)."""
    rng = np.random.default_rng(m)
    N = 50
    Xf = rng.standard_normal((m, N))
    rowptr, col, w = synth.identity_operator(m)
    r = np.ones(m)
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N))
    _, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-12, max_iter=400,
                              keep_iterates=True)
    Zhat, D = info["Zhat"], info["D"]
    S = Zhat @ Zhat.T / (N - 1) + np.eye(m)
    lam = np.linalg.eigvalsh(S)
    q = (math.sqrt(lam[-1] / lam[0]) - 1) / (math.sqrt(lam[-1] / lam[0]) + 1)
    Zs = np.linalg.solve(S, D)
    snorm = lambda E_: np.sqrt(np.einsum("ij,ij->j", E_, S @ E_))
    e0 = snorm(Zs - info["iterates"][0])
    for it, Zr in enumerate(info["iterates"][1:], start=1):
        er = snorm(Zs - Zr)
        assert np.all(er <= 2 * q ** it * e0 * (1 + 1e-9) + 1e-12 * e0)


def test_cg_converges_to_exact_and_stops_on_tolerance():
    p = synth.workload("grf512_N64_m65536", 5, scale=16)
    E = oracle.obs_perturbations(5, 2, p.r, p.N)
    ref = oracle.enkf_alg1(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    for tol in (1e-4, 1e-8, 1e-12):
        Xa, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, tol=tol)
        assert info["relres"].max() <= tol
        Zhat, D = info["Zhat"], info["D"]
        true = D - oracle.S_matvec(Zhat, p.r, info["Z"])
        rel_true = np.linalg.norm(true, axis=0) / np.linalg.norm(D, axis=0)
        assert rel_true.max() <= 10 * tol
    assert oracle.rel_frobenius(Xa, ref) < 1e-9


def test_zero_innovation_column_gives_zero_solution():
    Xf, rowptr, col, w, r, y, E = _tiny_problem(30, 6, 10, 12)
    Z = oracle.apply_H(rowptr, col, w, Xf)
    E = E.copy()
    E[:, 2] = Z[:, 2] - y        # makes d_2 = 0
    _, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-10)
    assert np.all(info["Z"][:, 2] == 0.0) and info["iters"][2] == 0


def test_reduced_cg_converges_within_N_steps_to_alg2():
    p = synth.workload("grf512_N64_m65536", 6, scale=16)
    E = oracle.obs_perturbations(6, 0, p.r, p.N)
    ref = oracle.enkf_alg2(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    Xa, info = oracle.cgd_enkf_reduced(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, tol=1e-14,
                                       max_iter=p.N + 1)
    assert info["iters"].max() <= p.N + 1
    assert oracle.rel_frobenius(Xa, ref) < 1e-10


def test_reduced_one_step_error_tends_to_one_as_m_grows():
    """Table 5's trend for CGD-EnKF-Reduced with one CG step: the relative error against
    EnKF-Reduced approaches 1 as the observation count grows (the eigenvalues of
    I + P^T P outside the constant direction grow with m)."""
    errs = []
    for m in (64, 1024, 16384):
        rng = np.random.default_rng(m)
        n, N = m, 20
        xt = rng.standard_normal(n)
        Xf = xt[:, None] + 0.1 * rng.standard_normal((n, N)) + 2.0
        rowptr, col, w = synth.identity_operator(n)
        r = np.full(m, 0.09)
        y = xt + 2.0 + 0.3 * rng.standard_normal(m)
        ref = oracle.enkf_alg2(Xf, rowptr, col, w, r, y)
        Xa, _ = oracle.cgd_enkf_reduced(Xf, rowptr, col, w, r, y, fixed_iters=1)
        errs.append(oracle.rel_frobenius(Xa, ref))
    assert errs[0] < errs[1] < errs[2] and errs[2] > 0.9


def test_senkf_differs_from_enkf_but_equals_it_for_uncorrelated_single_rows():
    Xf, rowptr, col, w, r, y, E = _tiny_problem(40, 10, 15, 13)
    a = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    s = oracle.senkf_alg3(Xf, rowptr, col, w, r, y, E)
    assert oracle.rel_frobenius(s, a) > 1e-6


def test_senkf_equals_enkf_when_observed_anomalies_are_orthogonal():
    # Algorithm 3 replaces S by its diagonal; when the rows of Z-hat are mutually orthogonal
    # (Hadamard rows 1..7 are zero-mean and orthogonal), HA HA^T is diagonal, S equals its
    # diagonal and the sEnKF analysis is the exact EnKF analysis (Sec. 2.2 / Appendix A).
    Hd = np.array([[1.0]])
    for _ in range(3):
        Hd = np.block([[Hd, Hd], [Hd, -Hd]])
    rng = np.random.default_rng(17)
    n, N = 12, 8
    Xf = rng.standard_normal((n, 1)) + 0.2 * rng.standard_normal((n, N))
    obs = [2, 5, 7, 10]
    for q, a in enumerate(obs):   # observed states: mean + scaled Hadamard row (distinct rows)
        Xf[a] = 1.5 + (0.3 + 0.1 * q) * Hd[q + 1]
    rowptr = np.arange(len(obs) + 1, dtype=np.int32)
    col = np.array(obs, np.int32)
    w = np.ones(len(obs))
    r = np.array([0.04, 0.5, 0.2, 1.3])
    y = rng.standard_normal(len(obs))
    E = 0.1 * rng.standard_normal((len(obs), N))
    _, _, _, _, Zhat = oracle.ensemble_stats(Xf, rowptr, col, w)
    G = Zhat @ Zhat.T
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-12
    a = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E)
    s = oracle.senkf_alg3(Xf, rowptr, col, w, r, y, E)
    assert np.max(np.abs(s - a)) < 1e-12
    assert oracle.rel_frobenius(a, Xf) > 1e-2     # the analysis does move the ensemble


# ---------------------------------------------------------------- generator pins
def test_philox_known_answer_vectors():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(*v[:4], *v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_perturbations_are_normal_with_variance_r():
    m, N = 4000, 64
    r = np.linspace(0.25, 2.0, m)
    E = oracle.obs_perturbations(1234, 0, r, N)
    xi = E / np.sqrt(r)[:, None]
    assert abs(xi.mean()) < 0.01
    assert abs(xi.var() - 1.0) < 0.01
    assert abs(np.mean(xi ** 4) - 3.0) < 0.05          # Gaussian kurtosis
    assert abs(np.corrcoef(xi[:, 0::2].ravel(), xi[:, 1::2].ravel())[0, 1]) < 0.01
    # counter and seed select independent streams; odd N drops the last sine draw
    assert not np.allclose(E, oracle.obs_perturbations(1234, 1, r, N))
    assert not np.allclose(E, oracle.obs_perturbations(1235, 0, r, N))
    assert np.array_equal(oracle.obs_perturbations(1234, 0, r, 63), E[:, :63])


def test_grf_generator_variance_and_correlation():
    x = synth.grf_fields(64, 4.0, 400, np.random.default_rng(0))
    assert abs(x.var() - 1.0) < 0.03
    f = x.T.reshape(400, 64, 64)
    lag = np.mean(f[:, :, :-3] * f[:, :, 3:])
    assert abs(lag - math.exp(-9.0 / 32.0)) < 0.03


def test_perturbation_definition_on_known_answer_block():
    """Row 0, members 0 and 1 with seed 0, counter 0 use Philox counter (0, 0, 0, 0) and key
    (0, 0): the first known-answer block. Evaluate the 53-bit uniforms and Box-Muller of
    the generator's definition with Python integers and the math module."""
    w0, w1, w2, w3 = 0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8
    u1 = (((w0 << 21) | (w1 >> 11)) + 0.5) / 2.0 ** 53
    u2 = ((w2 << 21) | (w3 >> 11)) / 2.0 ** 53
    rho = math.sqrt(-2.0 * math.log(u1))
    xi = [rho * math.cos(2 * math.pi * u2), rho * math.sin(2 * math.pi * u2)]
    E = oracle.obs_perturbations(0, 0, np.array([2.0]), 2)
    assert np.allclose(E[0], np.sqrt(2.0) * np.array(xi), rtol=1e-14, atol=0)
