"""Gaussian random fields on a periodic square grid (input generator).

Covariance convention: C(d) = exp(-d^2 / (2 l^2)), unit variance, d the distance on the
torus, separable in the two grid axes. Sampling is by circulant embedding: a stationary
covariance on the torus is diagonalised by the 2-D DFT, so with white noise w,
x = IDFT(sqrt(lam) * DFT(w)) has covariance exactly C when every eigenvalue lam >= 0
(negative round-off eigenvalues are clipped to zero).
"""
import numpy as np


def periodic_sqexp_eigenvalues(side: int, ell: float) -> np.ndarray:
    """Eigenvalues (rfft2 layout, shape (side, side//2+1)) of the separable periodic
    squared-exponential covariance on a side x side torus."""
    k = np.arange(side)
    d = np.minimum(k, side - k).astype(np.float64)
    c1 = np.exp(-(d * d) / (2.0 * ell * ell))
    lam1 = np.fft.fft(c1).real
    lam1 = np.clip(lam1, 0.0, None)
    lam = np.outer(lam1, lam1[: side // 2 + 1])
    return lam


def grf_fields(side: int, ell: float, count: int, rng: np.random.Generator,
               dtype=np.float64, chunk: int = 16) -> np.ndarray:
    """`count` independent zero-mean unit-variance fields, returned as an (side*side, count)
    C-contiguous array: grid point (row-major y*side+x) major, field index fastest, which is
    the [n][N] ensemble layout the analysis uses."""
    n = side * side
    out = np.empty((n, count), dtype=dtype)
    sq = np.sqrt(periodic_sqexp_eigenvalues(side, ell))
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        w = rng.standard_normal((c1 - c0, side, side))
        x = np.fft.irfft2(np.fft.rfft2(w) * sq, s=(side, side))
        out[:, c0:c1] = x.reshape(c1 - c0, n).T
    return out
