"""FP64 CPU oracle of the EnKF analysis step (test infrastructure only).

Notation: the library's letters are used (state dimension n, observation dimension m,
ensemble size N); the paper writes m, p, N. X_f is (n, N) with the member index fastest,
H is a CSR index-and-weight operator (rowptr, col, w), R = diag(r).

Every function follows a passage of the paper (Lee, Liu, Valyou, Zikatanov, "A Conjugate
Gradient Formulation of the EnKF Algorithm"):
  * ensemble statistics and Z-hat .......... Sec. 2.3, Eq. Zhat_def and Eq. Psi_zz
  * exact EnKF, dense Cholesky ............. Algorithm 1 (Sec. 5)
  * exact EnKF, N x N (Woodbury/Duncan) .... Algorithm 2, Eqs. LL-0, LL, LL-2 (Sec. 5.1)
  * CGD-EnKF ............................... Sec. 3.1-3.3, Eq. K_KF_T_rewrite, Eq. matvec_decomp
  * CGD-EnKF-Reduced ....................... Sec. 5.2 (Algorithm 2 with the N x N inverse
                                             replaced by CG on I + P^T P)
  * serial EnKF, matrix form ............... Algorithm 3 (Appendix A)
  * Kalman filter analysis ................. Sec. 2.2, Eqs. KF_analysis_1/2
  * relative Frobenius error ............... Eq. rel_frob (Sec. 6.2.2)
  * tridiagonal R (Example 2's noise model) . Sec. 5.3 (parallel complexity under
                                             tridiagonal Toeplitz R) and Sec. 6.2: every
                                             function below takes the off-diagonal r_off
                                             (R_{i,i+1} = R_{i+1,i} = r_off[i]) beside the
                                             diagonal r; r_off = None is diagonal R

Readings where the paper is silent (stated once here, used throughout):
  * Perturbed observations: the paper's EnKF is unperturbed (Remark after Eq. Psi_zz); the
    library perturbs with E (m, N), E = 0 reproduces the paper exactly. The innovation is
    D = Y + E - Z with Y = y 1^T.
  * CGD-EnKF solves S Z = D for the N innovation columns, S = HA HA^T/(N-1) + R (HA = Z-hat),
    then X_a = X_f + A (HA^T Z)/(N-1). At convergence this equals the paper's K^T form
    (Eq. K_KF_T_rewrite), which has n right-hand sides instead of N.
  * CG: N independent Hestenes-Stiefel recurrences (one per column, each with its own
    alpha_j, beta_j) sharing each matvec; start Z0 = 0 unless given; column j stops when
    ||r_j||_2 <= tol * ||d_j||_2 (d_j = 0 gives z_j = 0); `fixed_iters` > 0 runs exactly
    that many steps on every column that has not reached a zero residual.
  * CGD-EnKF-Reduced with E: X_a = X_f (I + P^T P)^{-1} [I + P^T L^{-1}((y - zbar) 1^T + E)],
    which Algorithm 2's derivation gives when Y - Z is replaced by Y + E - Z.
  * Tridiagonal R: its Cholesky factor L (R = L L^T) is lower bidiagonal and is computed by
    the banded Cholesky recurrence (the paper notes c_R = O(p), Sec. 5.3); R_N = (N-1) R has
    the factor sqrt(N-1) L, so P = L^{-1} Z-hat / sqrt(N-1) takes one bidiagonal forward
    substitution per column.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def apply_H(rowptr, col, w, X):
    """Z = H X for the CSR operator (Sec. 2.3: Z = H X^f)."""
    m = len(rowptr) - 1
    H = sp.csr_matrix((np.asarray(w, np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(m, X.shape[0]))
    return np.asarray(H @ X)


def ensemble_stats(Xf, rowptr, col, w):
    """Sec. 2.3: ensemble mean xbar, anomalies A = X_f - xbar 1^T, predicted observations
    Z = H X_f, their mean zbar = Z 1 / N, and Z-hat = Z - zbar 1^T (Eq. Zhat_def)."""
    Xf = np.asarray(Xf, dtype=np.float64)
    N = Xf.shape[1]
    xbar = Xf.sum(axis=1) / N
    A = Xf - xbar[:, None]
    Z = apply_H(rowptr, col, w, Xf)
    zbar = Z.sum(axis=1) / N
    Zhat = Z - zbar[:, None]
    return xbar, A, Z, zbar, Zhat


def innovations(y, Z, E=None):
    """D = Y + E - Z with Y = y 1^T (Sec. 2.3, the update X^a = X^f + K(Y - Z), with the
    perturbations E added)."""
    D = np.asarray(y, np.float64)[:, None] - Z
    if E is not None:
        D = D + E
    return D


def S_matvec(Zhat, r, V, r_off=None):
    """S V = Z-hat (Z-hat^T V)/(N-1) + R V: the three stages of Eq. matvec_decomp (stage 3 a
    diagonal scaling, or the tridiagonal product for Example 2's R)."""
    N = Zhat.shape[1]
    if r_off is None:
        return Zhat @ (Zhat.T @ V) / (N - 1) + np.asarray(r)[:, None] * V
    return Zhat @ (Zhat.T @ V) / (N - 1) + R_apply(r, r_off, V)


def R_apply(r, r_off, V):
    """R V for R = diag(r) (r_off None) or the symmetric tridiagonal R with diagonal r and
    off-diagonal r_off (R_{i,i+1} = R_{i+1,i} = r_off[i], length m-1)."""
    V = np.asarray(V, np.float64)
    r = np.asarray(r, np.float64)
    out = r[:, None] * V if V.ndim == 2 else r * V
    if r_off is not None:
        e = np.asarray(r_off, np.float64)
        if V.ndim == 2:
            e = e[:, None]
        out[:-1] += e * V[1:]
        out[1:] += e * V[:-1]
    return out


def R_dense(r, r_off=None):
    """The m x m matrix R (dense; small problems only)."""
    R = np.diag(np.asarray(r, np.float64))
    if r_off is not None:
        e = np.asarray(r_off, np.float64)
        R += np.diag(e, 1) + np.diag(e, -1)
    return R


def tridiag_cholesky(r, r_off):
    """Lower bidiagonal L with L L^T = R for the tridiagonal R: L[i,i] = l[i],
    L[i,i-1] = lo[i] (lo[0] = 0), by the banded Cholesky recurrence
    l[0] = sqrt(r[0]); lo[i] = r_off[i-1] / l[i-1], l[i] = sqrt(r[i] - lo[i]^2).
    Raises ValueError if R is not positive definite."""
    r = np.asarray(r, np.float64)
    e = np.asarray(r_off, np.float64)
    m = r.size
    l = np.empty(m)
    lo = np.zeros(m)
    l[0] = np.sqrt(r[0])
    for i in range(1, m):
        lo[i] = e[i - 1] / l[i - 1]
        d = r[i] - lo[i] * lo[i]
        if not d > 0.0:
            raise ValueError("R is not positive definite")
        l[i] = np.sqrt(d)
    return l, lo


def L_solve(r, r_off, B):
    """L^{-1} B for R = L L^T: r / sqrt for diagonal R, else one bidiagonal forward
    substitution per column (scipy's banded solver as the library step)."""
    B = np.asarray(B, np.float64)
    if r_off is None:
        d = np.sqrt(np.asarray(r, np.float64))
        return B / (d[:, None] if B.ndim == 2 else d)
    l, lo = tridiag_cholesky(r, r_off)
    ab = np.vstack([l, np.concatenate([lo[1:], [0.0]])])   # (l, u) = (1, 0) banded storage
    return sla.solve_banded((1, 0), ab, B)


def L_apply(r, r_off, B):
    """L B for R = L L^T (diagonal: sqrt(r) B)."""
    B = np.asarray(B, np.float64)
    if r_off is None:
        d = np.sqrt(np.asarray(r, np.float64))
        return d[:, None] * B if B.ndim == 2 else d * B
    l, lo = tridiag_cholesky(r, r_off)
    out = (l[:, None] * B) if B.ndim == 2 else l * B
    out[1:] += (lo[1:, None] * B[:-1]) if B.ndim == 2 else lo[1:] * B[:-1]
    return out


def enkf_alg1(Xf, rowptr, col, w, r, y, E=None, r_off=None):
    """Algorithm 1 (exact EnKF, matrix form), generalised by E:
    X_a = X_f + X_f Z-hat^T (Z-hat Z-hat^T + R_N)^{-1} ((y - zbar) 1^T - Z-hat + E),
    R_N = (N-1) R, solved with a dense Cholesky factorisation of the m x m matrix."""
    Xf = np.asarray(Xf, np.float64)
    N = Xf.shape[1]
    xbar, A, Z, zbar, Zhat = ensemble_stats(Xf, rowptr, col, w)
    Yhat = (np.asarray(y) - zbar)[:, None] * np.ones((1, N))
    rhs = Yhat - Zhat
    if E is not None:
        rhs = rhs + E
    C = Zhat @ Zhat.T + (N - 1) * R_dense(r, r_off)
    cf = sla.cho_factor(C, lower=True)
    sol = sla.cho_solve(cf, rhs)
    # the product X_f Z-hat^T sol, associated so that the intermediate stays small
    if Xf.shape[0] * len(r) <= N * N:
        return Xf + (Xf @ Zhat.T) @ sol
    return Xf + Xf @ (Zhat.T @ sol)


def enkf_alg2(Xf, rowptr, col, w, r, y, E=None, r_off=None):
    """Algorithm 2 (EnKF-Reduced), generalised by E:
    R_N = L L^T (L = diag(sqrt((N-1) r)) for diagonal R, sqrt(N-1) times the bidiagonal
    Cholesky factor of R for tridiagonal R), P = L^{-1} Z-hat,
    X_a = X_f (I + P^T P)^{-1} [I + P^T L^{-1} ((y - zbar) 1^T + E)]; the N x N matrix is
    factorised by Cholesky."""
    Xf = np.asarray(Xf, np.float64)
    N = Xf.shape[1]
    xbar, A, Z, zbar, Zhat = ensemble_stats(Xf, rowptr, col, w)
    sN = np.sqrt(N - 1.0)
    P = L_solve(r, r_off, Zhat) / sN
    G = np.eye(N) + P.T @ P
    Yt = (np.asarray(y) - zbar)[:, None] * np.ones((1, N))
    if E is not None:
        Yt = Yt + E
    M = np.eye(N) + P.T @ (L_solve(r, r_off, Yt) / sN)
    return Xf @ sla.cho_solve(sla.cho_factor(G, lower=True), M)


def enkf_exact(Xf, rowptr, col, w, r, y, E=None, m_dense=8192, r_off=None):
    """The exact analysis: Algorithm 1 (dense m x m Cholesky) when m <= m_dense, otherwise
    Algorithm 2 (N x N Cholesky), which gives the same result (Eqs. LL-0 to LL-2)."""
    if len(r) <= m_dense:
        return enkf_alg1(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    return enkf_alg2(Xf, rowptr, col, w, r, y, E, r_off=r_off)


def _cg_columns(matvec, B, tol, max_iter, fixed_iters=0, X0=None, keep_iterates=False):
    """N independent conjugate-gradient recurrences (Hestenes-Stiefel, Sec. 3.1) for
    M X = B, one per column, sharing each application of M. Returns X, iteration counts,
    final recursive relative residuals ||r_j|| / ||b_j|| and optionally every iterate."""
    B = np.asarray(B, np.float64)
    ncol = B.shape[1]
    X = np.zeros_like(B) if X0 is None else np.array(X0, np.float64, copy=True)
    R = B - matvec(X) if X0 is not None else B.copy()
    P = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    bnorm = np.sqrt(np.einsum("ij,ij->j", B, B))
    iters = np.zeros(ncol, dtype=np.int64)
    limit = fixed_iters if fixed_iters > 0 else max_iter
    if fixed_iters > 0:
        active = rr > 0
    else:
        active = np.sqrt(rr) > tol * bnorm
    iterates = [X.copy()] if keep_iterates else None
    for _ in range(limit):
        if not active.any():
            break
        Q = matvec(P)
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        X += alpha * P
        R -= alpha * Q
        rr_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        P = np.where(active, R + beta * P, P)
        rr = np.where(active, rr_new, rr)
        iters += active
        if fixed_iters > 0:
            active = active & (rr > 0)
        else:
            active = active & (np.sqrt(rr) > tol * bnorm)
        if keep_iterates:
            iterates.append(X.copy())
    relres = np.sqrt(rr) / np.where(bnorm > 0, bnorm, 1.0)
    return X, iters, relres, iterates


def cgd_enkf(Xf, rowptr, col, w, r, y, E=None, tol=1e-10, max_iter=1000, fixed_iters=0,
             Z0=None, keep_iterates=False, r_off=None):
    """CGD-EnKF (Sec. 3.2, Fig. 2) in the N-right-hand-side form: solve S Z = D by CG with
    the matvec of Eq. matvec_decomp, then X_a = X_f + A (Z-hat^T Z)/(N-1).
    Returns (X_a, info) with info = dict(Z, iters, relres, W, iterates)."""
    Xf = np.asarray(Xf, np.float64)
    N = Xf.shape[1]
    xbar, A, Z, zbar, Zhat = ensemble_stats(Xf, rowptr, col, w)
    D = innovations(y, Z, E)
    Zs, iters, relres, its = _cg_columns(lambda V: S_matvec(Zhat, r, V, r_off), D, tol, max_iter,
                                         fixed_iters, Z0, keep_iterates)
    W = Zhat.T @ Zs / (N - 1)
    return Xf + A @ W, dict(Z=Zs, iters=iters, relres=relres, W=W, D=D, Zhat=Zhat,
                            iterates=its)


def cgd_enkf_reduced(Xf, rowptr, col, w, r, y, E=None, tol=1e-10, max_iter=1000,
                     fixed_iters=0, r_off=None):
    """CGD-EnKF-Reduced (Sec. 5.2): Algorithm 2 with (I + P^T P)^{-1} applied by CG
    ("block CGD", N independent columns) to the N right-hand sides
    M = I + P^T L^{-1}((y - zbar) 1^T + E); X_a = X_f V with V the CG solution.
    Returns (X_a, info) with info = dict(V, iters, relres, G, M)."""
    Xf = np.asarray(Xf, np.float64)
    N = Xf.shape[1]
    xbar, A, Z, zbar, Zhat = ensemble_stats(Xf, rowptr, col, w)
    sN = np.sqrt(N - 1.0)
    P = L_solve(r, r_off, Zhat) / sN
    G = np.eye(N) + P.T @ P
    Yt = (np.asarray(y) - zbar)[:, None] * np.ones((1, N))
    if E is not None:
        Yt = Yt + E
    M = np.eye(N) + P.T @ (L_solve(r, r_off, Yt) / sN)
    V, iters, relres, _ = _cg_columns(lambda U: G @ U, M, tol, max_iter, fixed_iters)
    return Xf @ V, dict(V=V, iters=iters, relres=relres, G=G, M=M)


def senkf_alg3(Xf, rowptr, col, w, r, y, E=None, r_off=None):
    """Algorithm 3 (serial EnKF, matrix form, Appendix A), generalised by E:
    X_a = X_f + X_f Z-hat^T [diag(Z-hat Z-hat^T + R_N)]^{-1} (Y + E - Z). Only the diagonal
    of R_N enters, so r_off (a tridiagonal R's off-diagonal) does not change the result."""
    Xf = np.asarray(Xf, np.float64)
    N = Xf.shape[1]
    xbar, A, Z, zbar, Zhat = ensemble_stats(Xf, rowptr, col, w)
    dg = np.einsum("ij,ij->i", Zhat, Zhat) + (N - 1) * np.asarray(r, np.float64)
    return Xf + Xf @ (Zhat.T @ (innovations(y, Z, E) / dg[:, None]))


def kalman_analysis(xf, Pf, Hd, R, y):
    """Kalman filter analysis (Sec. 2.2): S = H P H^T + R, K = P H^T S^{-1},
    x_a = x_f + K (y - H x_f), P_a = (I - K H) P. Dense matrices; small problems only."""
    S = Hd @ Pf @ Hd.T + R
    K = np.linalg.solve(S.T, (Pf @ Hd.T).T).T
    xa = xf + K @ (y - Hd @ xf)
    Pa = (np.eye(Pf.shape[0]) - K @ Hd) @ Pf
    return xa, Pa, K


def rel_frobenius(X, Xref):
    """Eq. rel_frob: ||X - X_ref||_F / ||X_ref||_F."""
    X = np.asarray(X, np.float64)
    Xref = np.asarray(Xref, np.float64)
    return float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))
