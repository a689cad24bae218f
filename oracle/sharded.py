"""Row-block distributed CGD-EnKF on CPU ranks (test infrastructure only).

The paper's parallel form of the method (Sec. 3.3): every processor q owns a contiguous
block of observation rows of each distributed matrix and vector (Z-hat = HA, D, the CG
iterate, residual and direction), and the matvec of Eq. matvec_decomp runs in three stages:
(1) the local contribution HA_q^T d_q to HA^T d (N x N for the N columns), summed over the
processors (an allreduce), (2) the local rows of HA (HA^T d)/(N-1), (3) the local rows of
R d (diagonal R: no communication; tridiagonal R: the neighbouring processors' boundary
entries of d). The CG scalars need column sums over all rows: (p, S p) is ||HA^T p||^2/(N-1)
+ p^T R p, and (r, r) for alpha, beta and the stopping rule, each summed by an allreduce.
W = HA^T Z/(N-1) is summed the same way and replicated, and each processor updates its own
block of state rows, X_a = X_f + A W. With exact sums the result equals the single-process
CG (`oracle.cgd_enkf`) up to the order of the floating-point additions.

`allreduce(array)` returns the element-wise sum of `array` over all processors (every caller
gets the same result); `rank` and `size` name this processor and the processor count.
"""
import numpy as np

from .enkf import ensemble_stats, innovations


def row_block(count, rank, size):
    """The contiguous block [lo, hi) of `count` rows owned by processor `rank` of `size`."""
    per = -(-count // size)
    lo = min(count, rank * per)
    return lo, min(count, lo + per)


def _halo(v, lo, hi, m, rank, size, allreduce):
    """The rows lo-1 and hi of v (N columns) owned by the neighbouring processors (zeros past
    the ends): every processor publishes its first and last row in its own slots of a
    (2 size, N) array and one allreduce delivers all of them."""
    N = v.shape[1]
    buf = np.zeros((2 * size, N))
    if hi > lo:
        buf[2 * rank] = v[0]
        buf[2 * rank + 1] = v[-1]
    buf = allreduce(buf)
    below = np.zeros(N)
    above = np.zeros(N)
    if lo > 0:        # the processor that owns row lo-1 published it as its last row
        q = next(k for k in range(size) if row_block(m, k, size)[1] == lo)
        below = buf[2 * q + 1]
    if hi < m:        # the processor that owns row hi published it as its first row
        q = next(k for k in range(size) if row_block(m, k, size)[0] == hi)
        above = buf[2 * q]
    return below, above


def _local_R(v, r, r_off, lo, hi, m, rank, size, allreduce):
    """Stage 3: the local rows of R v (R diagonal, or tridiagonal with off-diagonal r_off)."""
    out = r[lo:hi, None] * v
    if r_off is None:
        return out
    below, above = _halo(v, lo, hi, m, rank, size, allreduce)
    if hi > lo:
        e = r_off
        up = np.vstack([v[1:], above[None, :]])          # rows lo+1 .. hi
        dn = np.vstack([below[None, :], v[:-1]])         # rows lo-1 .. hi-2
        e_up = e[lo:hi][:, None] if hi < m else np.concatenate([e[lo:hi - 1], [0.0]])[:, None]
        e_dn = np.concatenate([[e[lo - 1]] if lo > 0 else [0.0], e[lo:hi - 1]])[:, None]
        out = out + e_up * up + e_dn * dn
    return out


def cgd_enkf_rowblock(Xf, rowptr, col, w, r, y, rank, size, allreduce, E=None, tol=1e-10,
                      max_iter=1000, fixed_iters=0, r_off=None):
    """CGD-EnKF (plain CG on S Z = D, N columns) with the observation rows and the state rows
    split in row blocks over `size` processors (Sec. 3.3). Every processor passes the full
    inputs and works on its own blocks. Returns (the processor's block of X_a rows, (lo, hi)
    of its state rows, info with the replicated W and the CG iteration counts)."""
    Xf = np.asarray(Xf, np.float64)
    n, N = Xf.shape
    m = len(r)
    r = np.asarray(r, np.float64)
    # this processor's observation rows and the ensemble statistics they need (row-local)
    lo, hi = row_block(m, rank, size)
    sub = slice(lo, hi)
    rp = np.asarray(rowptr)[lo:hi + 1] - rowptr[lo]
    cols = np.asarray(col)[rowptr[lo]:rowptr[hi]]
    ws = np.asarray(w)[rowptr[lo]:rowptr[hi]]
    _, _, Z, zbar, HA = ensemble_stats(Xf, rp, cols, ws)
    D = innovations(np.asarray(y)[sub], Z, None if E is None else np.asarray(E)[sub])

    def dots(a, b):                      # column sums over all observation rows
        return allreduce(np.einsum("ij,ij->j", a, b))

    def matvec(V):
        T = allreduce(HA.T @ V)          # stage 1 (+ allreduce)
        return HA @ T / (N - 1) + _local_R(V, r, r_off, lo, hi, m, rank, size, allreduce), T

    X = np.zeros_like(D)
    R_ = D.copy()
    P = R_.copy()
    rr = dots(R_, R_)
    bn = np.sqrt(rr)
    iters = np.zeros(N, dtype=np.int64)
    active = (rr > 0) if fixed_iters > 0 else (np.sqrt(rr) > tol * bn)
    limit = fixed_iters if fixed_iters > 0 else max_iter
    for _ in range(limit):
        if not active.any():
            break
        Q, _ = matvec(P)                 # stages 2 and 3
        pq = dots(P, Q)
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        X += alpha * P
        R_ -= alpha * Q
        rr_new = dots(R_, R_)
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        P = np.where(active, R_ + beta * P, P)
        rr = np.where(active, rr_new, rr)
        iters += active
        active = active & ((rr > 0) if fixed_iters > 0 else (np.sqrt(rr) > tol * bn))
    W = allreduce(HA.T @ X) / (N - 1)
    # the update of this processor's block of state rows (W is replicated)
    slo, shi = row_block(n, rank, size)
    Xb = Xf[slo:shi]
    A = Xb - Xb.mean(axis=1, keepdims=True)
    return Xb + A @ W, (slo, shi), dict(W=W, iters=iters)
