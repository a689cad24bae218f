"""Oracle side of the observation-perturbation generator (test infrastructure).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): a 4x32-bit counter and a 2x32-bit
key go through 10 rounds; each round multiplies counter words 0 and 2 by the constants
0xD2511F53 and 0xCD9E8D57 into 64-bit products, and the new counter is
(hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)); between rounds the key
is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85), mod 2^32.

Perturbation layout (the definition both implementations follow):
  element (i, j) of E (observation i, member j) uses counter (i, j >> 1, ctr_lo, ctr_hi)
  and key (seed_lo, seed_hi); output words (w0, w1, w2, w3) give two 53-bit uniforms
  u1 = ((w0 << 21 | w1 >> 11) + 0.5) / 2^53 in (0, 1) and u2 = (w2 << 21 | w3 >> 11) / 2^53,
  and Box-Muller gives xi = sqrt(-2 ln u1) * cos(2 pi u2) for even j, * sin(2 pi u2) for
  odd j; E_ij = sqrt(r_i) * xi_ij, so each column of E is a draw from N(0, R) with R
  diagonal (the perturbed-observation EnKF's E ~ N(0, R)).
"""
import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. Inputs are integer arrays (broadcastable) holding 32-bit
    values; returns four uint64 arrays holding the 32-bit output words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> _S32) ^ c1 ^ k0, p1 & _MASK, (p0 >> _S32) ^ c3 ^ k1, p0 & _MASK)
    return c0, c1, c2, c3


def uniform53_pair(w0, w1, w2, w3):
    x1 = (w0 << np.uint64(21)) | (w1 >> np.uint64(11))
    x2 = (w2 << np.uint64(21)) | (w3 >> np.uint64(11))
    u1 = (x1.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = x2.astype(np.float64) * 2.0 ** -53
    return u1, u2


def obs_perturbations(seed: int, counter: int, r: np.ndarray, N: int, r_off=None) -> np.ndarray:
    """E (m, N) with column j ~ N(0, R), drawn as defined in the module docstring: the
    standard normals xi scaled by sqrt(r) (diagonal R), or E = L xi with L the bidiagonal
    Cholesky factor of a tridiagonal R (diagonal r, off-diagonal r_off)."""
    m = r.shape[0]
    i = np.arange(m, dtype=np.uint64)[:, None]
    q = np.arange((N + 1) // 2, dtype=np.uint64)[None, :]
    w = philox4x32_10(i, q, counter & 0xFFFFFFFF, (counter >> 32) & 0xFFFFFFFF,
                      seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1, u2 = uniform53_pair(*w)
    rho = np.sqrt(-2.0 * np.log(u1))
    theta = 6.283185307179586 * u2
    xi = np.empty((m, 2 * q.shape[1]))
    xi[:, 0::2] = rho * np.cos(theta)
    xi[:, 1::2] = rho * np.sin(theta)
    if r_off is None:
        return np.sqrt(r)[:, None] * xi[:, :N]
    from .enkf import L_apply
    return L_apply(r, r_off, xi[:, :N])
