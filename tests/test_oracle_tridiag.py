"""Pins of the oracle's tridiagonal-R paths (Example 2's observation noise: R tridiagonal
Toeplitz, diagonal sigma^2, off-diagonals sigma^2 rho; Sec. 5.3 and Sec. 6.2) to facts outside
the oracle: an explicit Gauss-Jordan inverse with the full R on tiny inputs, L L^T = R for the
bidiagonal factor, Algorithm 1 (m x m Cholesky) = Algorithm 2 (bidiagonal L) = converged CG,
the diagonal case as a special case, the covariance of the drawn perturbations, and the
CGD-EnKF-Reduced errors the paper prints in Table 5 (tests/golden)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gauss_jordan_inverse(M):
    n = len(M)
    a = [list(map(float, row)) + [1.0 if i == j else 0.0 for j in range(n)] for i, row in enumerate(M)]
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


def _brute_force(Xf, rowptr, col, w, r, r_off, y, E):
    """X_a = X_f + Psi_x (Psi_zz + R)^{-1} (Y + E - Z), every covariance an explicit sum and
    R the full tridiagonal matrix (Sec. 2.3 with Example 2's R), inverse by Gauss-Jordan."""
    n, N, m = len(Xf), len(Xf[0]), len(r)
    Z = [[0.0] * N for _ in range(m)]
    for i in range(m):
        for k in range(rowptr[i], rowptr[i + 1]):
            for j in range(N):
                Z[i][j] += w[k] * Xf[col[k]][j]
    xbar = [sum(Xf[a]) / N for a in range(n)]
    zbar = [sum(Z[i]) / N for i in range(m)]

    def R(i, k):
        if i == k:
            return r[i]
        if abs(i - k) == 1:
            return r_off[min(i, k)]
        return 0.0

    Psi_x = [[sum((Xf[a][j] - xbar[a]) * (Z[i][j] - zbar[i]) for j in range(N)) / (N - 1) for i in range(m)]
             for a in range(n)]
    Psi_z = [[sum((Z[i][j] - zbar[i]) * (Z[k][j] - zbar[k]) for j in range(N)) / (N - 1) + R(i, k)
              for k in range(m)] for i in range(m)]
    Sinv = _gauss_jordan_inverse(Psi_z)
    K = [[sum(Psi_x[a][k] * Sinv[k][i] for k in range(m)) for i in range(m)] for a in range(n)]
    innov = [[y[i] + E[i][j] - Z[i][j] for j in range(N)] for i in range(m)]
    return [[Xf[a][j] + sum(K[a][i] * innov[i][j] for i in range(m)) for j in range(N)] for a in range(n)]


def _tiny(n, N, m, seed):
    rng = np.random.default_rng(seed)
    Xf = rng.standard_normal((n, N)) + rng.standard_normal(n)[:, None]
    rowptr, col, w = [0], [], []
    for _ in range(m):
        k = int(rng.integers(1, 4))
        col += list(rng.choice(n, size=k, replace=False))
        w += list(rng.uniform(-1.5, 1.5, size=k))
        rowptr.append(len(col))
    r = rng.uniform(0.5, 1.5, size=m)
    # off-diagonals small enough for positive definiteness (diagonal dominance)
    r_off = rng.uniform(-0.45, 0.45, size=m - 1) * np.minimum(r[:-1], r[1:])
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N))
    return Xf, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(w), r, r_off, y, E


def test_bidiagonal_factor_reproduces_R_and_rejects_indefinite():
    for m in (1, 2, 7, 40):
        r = np.full(m, 0.09)
        e = np.full(m - 1, 0.09 * 0.2)
        l, lo = oracle.tridiag_cholesky(r, e)
        L = np.diag(l) + np.diag(lo[1:], -1)
        assert np.max(np.abs(L @ L.T - oracle.R_dense(r, e))) <= 1e-16
        B = np.random.default_rng(m).standard_normal((m, 3))
        assert np.max(np.abs(L @ oracle.L_solve(r, e, B) - B)) <= 1e-14
        assert np.max(np.abs(oracle.L_apply(r, e, B) - L @ B)) <= 1e-15
    with pytest.raises(ValueError):
        oracle.tridiag_cholesky(np.ones(3), np.array([0.9, 0.9]))   # eigenvalue 1 - 0.9 sqrt(2) < 0


@pytest.mark.parametrize("n,N,m,seed", [(5, 4, 3, 0), (6, 3, 5, 1), (4, 6, 4, 2), (7, 2, 6, 3)])
def test_alg1_tridiagonal_matches_gauss_jordan_brute_force(n, N, m, seed):
    Xf, rowptr, col, w, r, r_off, y, E = _tiny(n, N, m, seed)
    ref = np.array(_brute_force(Xf.tolist(), rowptr.tolist(), col.tolist(), w.tolist(), r.tolist(),
                                r_off.tolist(), y.tolist(), E.tolist()))
    got = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # and the diagonal R is the special case r_off = 0
    z = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E, r_off=np.zeros(m - 1))
    assert np.max(np.abs(z - oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E))) <= 1e-13


@pytest.mark.parametrize("n,N,m", [(30, 8, 12), (40, 20, 20), (200, 16, 150), (300, 40, 300)])
def test_alg2_bidiagonal_and_converged_cg_equal_alg1(n, N, m):
    Xf, rowptr, col, w, r, r_off, y, E = _tiny(n, N, m, n + N + m)
    a1 = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    a2 = oracle.enkf_alg2(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    assert oracle.rel_frobenius(a2, a1) < 1e-11
    cg, info = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, tol=1e-13, r_off=r_off)
    assert oracle.rel_frobenius(cg, a1) < 1e-10
    red, _ = oracle.cgd_enkf_reduced(Xf, rowptr, col, w, r, y, E, tol=1e-13, r_off=r_off)
    assert oracle.rel_frobenius(red, a1) < 1e-10


def test_cg_matvec_stage3_is_the_tridiagonal_product():
    rng = np.random.default_rng(4)
    m, N = 9, 3
    HA = rng.standard_normal((m, N))
    r = rng.uniform(1, 2, m)
    e = rng.uniform(-0.3, 0.3, m - 1)
    V = rng.standard_normal((m, 2))
    S = HA @ HA.T / (N - 1) + oracle.R_dense(r, e)
    assert np.max(np.abs(oracle.S_matvec(HA, r, V, e) - S @ V)) <= 1e-14


def test_perturbations_with_tridiagonal_R_have_covariance_R():
    m, N = 5, 20000
    r = np.full(m, 0.09)
    e = np.full(m - 1, 0.018)
    E = oracle.obs_perturbations(3, 1, r, N, r_off=e)
    C = E @ E.T / N
    assert np.max(np.abs(C - oracle.R_dense(r, e))) <= 5 * 0.09 * math.sqrt(2.0 / N)
    # the same standard normals as the diagonal draw: E = L xi with xi = diagonal draw / sqrt(r)
    xi = oracle.obs_perturbations(3, 1, np.ones(m), N)
    l, lo = oracle.tridiag_cholesky(r, e)
    assert np.max(np.abs(E - (np.diag(l) + np.diag(lo[1:], -1)) @ xi)) <= 1e-15


def _table5():
    rows = []
    with open(os.path.join(GOLDEN, "table5_cgd_enkf_reduced.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p, r, v = line.split()
                rows.append((int(p), int(r), float(v)))
    return rows


@pytest.mark.parametrize("p", [1000, 10000])
def test_table5_cgd_reduced_errors_reproduce_the_printed_values(p):
    """Example 2b: L96, H = I, N = 100, sigma = 0.3, rho = 0.2. The paper's seeds and states
    are unpublished, so the printed errors are matched within bands that the seed-to-seed
    spread of the workload covers: 5 % for r = 1, 2 (errors near 1 or 0.3), 25 % for r = 3,
    a factor 2.5 for r = 4, 5 (errors 1e-2 .. 1e-4, set by the smallest eigenvalues)."""
    P = synth.l96_tridiag_problem(p, 100, seed=1)
    ref = oracle.enkf_alg2(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, None, r_off=P.r_off)
    band = {1: 1.05, 2: 1.05, 3: 1.25, 4: 2.5, 5: 2.5}
    for pp, r, printed in _table5():
        if pp != p or r == 0:
            continue
        X, _ = oracle.cgd_enkf_reduced(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, None, fixed_iters=r, r_off=P.r_off)
        err = oracle.rel_frobenius(X, ref)
        assert abs(math.log(err / printed)) <= math.log(band[r]), (p, r, err, printed)


def test_table5_trends():
    """The trends Table 5 shows: at fixed p the error falls with r; at r = 1 it grows toward 1
    with p, at r = 5 it falls with p (the spectrum of I + P^T P clusters as p grows)."""
    errs = {}
    for p in (1000, 10000, 100000):
        P = synth.l96_tridiag_problem(p, 100, seed=2)
        ref = oracle.enkf_alg2(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, None, r_off=P.r_off)
        errs[p] = [oracle.rel_frobenius(oracle.cgd_enkf_reduced(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, None,
                                                                fixed_iters=r, r_off=P.r_off)[0], ref)
                   for r in range(1, 6)]
        assert all(a > b for a, b in zip(errs[p][:-1], errs[p][1:])), errs[p]
    assert errs[1000][0] < errs[10000][0] < errs[100000][0] < 1.0
    assert errs[1000][4] > errs[10000][4] > errs[100000][4]


def test_senkf_uses_only_the_diagonal_of_R():
    Xf, rowptr, col, w, r, r_off, y, E = _tiny(20, 6, 10, 9)
    a = oracle.senkf_alg3(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    b = oracle.senkf_alg3(Xf, rowptr, col, w, r, y, E)
    assert np.array_equal(a, b)
