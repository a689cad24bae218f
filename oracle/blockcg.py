"""Block conjugate gradients and the CG error bounds of the paper (test infrastructure only).

* Block CG (O'Leary 1980, "The block conjugate gradient algorithm and related methods"), the
  other reading of the paper's "block CGD" (Sec. 3.1, Table 2): the N right-hand sides of
  S Z = D share one block Krylov space, X_{k+1} = X_k + P_k a_k, R_{k+1} = R_k - S P_k a_k,
  P_{k+1} = Z_{k+1} + P_k b_k with the N x N coefficient matrices
  a_k = (P_k^T S P_k)^{-1} (Z_k^T R_k), b_k = (Z_k^T R_k)^{-1} (Z_{k+1}^T R_{k+1}), Z = M^{-1} R
  (M = I, or M = R for the preconditioned form). For S = HA HA^T/(N-1) + R the preconditioned
  operator is the identity plus a rank N-1 term, so the exact solution lies in a block Krylov
  space of two blocks.
* The energy-norm error bounds of Prop. 1 (classical, 2 ((sqrt k - 1)/(sqrt k + 1))^r) and
  Prop. 3 (Sec. 4): with the l unique eigenvalues outside [lambda_a, lambda_b] as sigma_0 and
  the rest as sigma_1, for r >= l,
      ||e_r||_S <= 2 C ((sqrt k_eff - 1)/(sqrt k_eff + 1))^(r - l) ||e_0||_S,
      C = max_{lambda in sigma_1} prod_{mu in sigma_0} |1 - lambda/mu|,  k_eff = lambda_b/lambda_a
  (the factor 2 outside the power, as in the proposition's statement).
"""
import numpy as np


def block_cg(matvec, B, tol=1e-10, max_iter=200, fixed_iters=0, precond=None):
    """Block CG for S X = B (all columns in one block). `precond(R)` applies M^{-1} (None: I).
    Returns (X, steps, final relative residual norms per column)."""
    B = np.asarray(B, np.float64)
    X = np.zeros_like(B)
    R = B.copy()
    Z = R if precond is None else precond(R)
    P = Z.copy()
    bn = np.linalg.norm(B, axis=0)
    bn = np.where(bn > 0, bn, 1.0)
    G = Z.T @ R
    steps = 0
    limit = fixed_iters if fixed_iters > 0 else max_iter
    while steps < limit:
        if fixed_iters == 0 and np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        Q = matvec(P)
        a = np.linalg.solve(P.T @ Q, G)
        X += P @ a
        R -= Q @ a
        Z = R if precond is None else precond(R)
        Gn = Z.T @ R
        steps += 1
        if fixed_iters == 0 and np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        b = np.linalg.solve(G, Gn)
        P = Z + P @ b
        G = Gn
    return X, steps, np.linalg.norm(R, axis=0) / bn


def energy_errors(S, B, iterates):
    """||x* - x_r||_S per iterate (columns averaged), x* = S^{-1} B from a dense solve."""
    Xs = np.linalg.solve(S, B)
    out = []
    for X in iterates:
        E = Xs - X
        out.append(float(np.mean(np.sqrt(np.einsum("ij,ij->j", E, S @ E)))))
    return np.array(out)


def _rate(kappa):
    s = np.sqrt(kappa)
    return (s - 1.0) / (s + 1.0)


def classical_bound(eigs, r):
    """Prop. 1: 2 ((sqrt(cond) - 1)/(sqrt(cond) + 1))^r (times ||e_0||_S)."""
    eigs = np.sort(np.asarray(eigs, np.float64))
    return 2.0 * _rate(eigs[-1] / eigs[0]) ** r


def prop3_bound(eigs, r, n_low, n_high, rel_unique=1e-10):
    """Prop. 3 with the n_low smallest and n_high largest unique eigenvalues as sigma_0 (times
    ||e_0||_S); None if r < l = n_low + n_high or sigma_1 would be empty."""
    u = np.sort(np.asarray(eigs, np.float64))
    # unique eigenvalues (equal within rel_unique)
    keep = np.concatenate([[True], np.diff(u) > rel_unique * u[1:]])
    u = u[keep]
    l = n_low + n_high
    if r < l or l >= u.size:
        return None
    mu = np.concatenate([u[:n_low], u[u.size - n_high:]])
    s1 = u[n_low:u.size - n_high]
    lam_a, lam_b = s1[0], s1[-1]
    C = max(float(np.prod(np.abs(1.0 - lam / mu))) for lam in s1)
    return 2.0 * C * _rate(lam_b / lam_a) ** (r - l)


def prop3_best(eigs, r, max_out=None):
    """The smallest Prop. 3 bound over the splits with l <= r outliers (at most max_out)."""
    best = None
    lim = r if max_out is None else min(r, max_out)
    for nl in range(0, lim + 1):
        for nh in range(0, lim + 1 - nl):
            b = prop3_bound(eigs, r, nl, nh)
            if b is not None and (best is None or b < best):
                best = b
    return best
