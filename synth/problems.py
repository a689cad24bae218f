"""Seeded analysis problems with the shapes of the paper's and the benchmark's workloads.

A problem is (X_f, H, r, y): the forecast ensemble X_f laid out (n, N) with the member
index fastest; H as a CSR "index-and-weight" observation operator (rowptr[m+1], col[nnz],
w[nnz]) with Z = H X_f row i = sum_k w_k X_f[col_k]; the diagonal of R as r[m]; the
observation y[m] = H x_t + v, v ~ N(0, R), from an independent truth x_t.

Seeds: numpy PCG64 streams keyed by (seed, stream id) with fixed stream ids (0 truth,
1 ensemble, 2 observation noise, 4 H subsample, 5 R). Stream 3 is reserved for the
analysis's own perturbations, which are not drawn here.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .grf import grf_fields
from .l96 import l96_rk4

STREAM_TRUTH, STREAM_ENSEMBLE, STREAM_OBSNOISE, STREAM_H, STREAM_R = 0, 1, 2, 4, 5


def _rng(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFF, stream, sub])


@dataclass
class Problem:
    Xf: np.ndarray            # (n, N) float64 or float32, C-contiguous
    rowptr: np.ndarray        # (m+1,) int32
    col: np.ndarray           # (nnz,) int32
    w: np.ndarray             # (nnz,) float64
    r: np.ndarray             # (m,) float64, > 0
    y: np.ndarray             # (m,) float64
    truth: np.ndarray = None  # (n,) float64
    meta: dict = field(default_factory=dict)
    r_off: np.ndarray = None  # (m-1,) float64: off-diagonal of a tridiagonal R, None = diagonal

    @property
    def n(self):
        return self.Xf.shape[0]

    @property
    def N(self):
        return self.Xf.shape[1]

    @property
    def m(self):
        return self.r.shape[0]


def subsample_operator(n: int, m: int, rng: np.random.Generator):
    """m distinct state indices drawn uniformly without replacement, sorted ascending,
    weight 1: a random point-subsample observation operator in CSR form."""
    idx = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    return np.arange(m + 1, dtype=np.int32), idx, np.ones(m, dtype=np.float64)


def identity_operator(n: int):
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n)


def every_kth_operator(n: int, k: int):
    idx = np.arange(0, n, k, dtype=np.int32)
    return np.arange(idx.size + 1, dtype=np.int32), idx, np.ones(idx.size)


def obs_variances(m: int, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(lo, hi, size=m)


def _observe(truth, rowptr, col, w, r, rng):
    m = r.shape[0]
    Hx = np.zeros(m)
    np.add.at(Hx, np.repeat(np.arange(m), np.diff(rowptr)), w * truth[col])
    return Hx + np.sqrt(r) * rng.standard_normal(m)


def grf_problem(side: int, ell: float, N: int, m: int, r_lo: float, r_hi: float,
                seed: int, dtype=np.float64, sub: int = 0, meta=None) -> Problem:
    """GRF forecast ensemble on a side x side torus (members i.i.d. zero-mean unit-variance
    fields), an independent GRF truth, a random m-point subsample H, r ~ U[r_lo, r_hi]."""
    n = side * side
    Xf = grf_fields(side, ell, N, _rng(seed, STREAM_ENSEMBLE, sub), dtype=dtype)
    truth = grf_fields(side, ell, 1, _rng(seed, STREAM_TRUTH, sub))[:, 0]
    rowptr, col, w = subsample_operator(n, m, _rng(seed, STREAM_H, sub))
    r = obs_variances(m, r_lo, r_hi, _rng(seed, STREAM_R, sub))
    y = _observe(truth, rowptr, col, w, r, _rng(seed, STREAM_OBSNOISE, sub))
    md = dict(side=side, ell=ell)
    md.update(meta or {})
    return Problem(np.ascontiguousarray(Xf), rowptr, col, w, r, y, truth, md)


# Workloads by what they are. `scale` shrinks the grid side (and the correlation length)
# by `scale` and the observation count by scale**2, keeping N.
WORKLOADS = {
    # 512x512 GRF (length 16 cells), N=64, 65,536 random point observations,
    # r ~ U[0.5, 1.5], CG relative-residual tolerance 1e-8
    "grf512_N64_m65536": dict(side=512, ell=16.0, N=64, m=65536, r=(0.5, 1.5), tol=1e-8),
    # 1024x1024 GRF (length 24), N=128, 262,144 observations, r ~ U[0.25, 1.0]
    "grf1024_N128_m262144": dict(side=1024, ell=24.0, N=128, m=262144, r=(0.25, 1.0),
                                 tol=1e-8),
}


def workload(name: str, seed: int, scale: int = 1, dtype=np.float64, sub: int = 0) -> Problem:
    c = WORKLOADS[name]
    side = c["side"] // scale
    m = c["m"] // (scale * scale)
    return grf_problem(side, c["ell"] / scale, c["N"], m, c["r"][0], c["r"][1], seed,
                       dtype=dtype, sub=sub, meta=dict(name=name, scale=scale, tol=c["tol"]))


def _tridiag_noise(sig2, off, rng, m):
    """A draw of N(0, R) for the symmetric tridiagonal Toeplitz R (diagonal sig2, off-diagonal
    off): v = C xi with C the lower bidiagonal factor of R (C C^T = R), from its recurrence."""
    xi = rng.standard_normal(m)
    v = np.empty(m)
    c_prev = math.sqrt(sig2)
    v[0] = c_prev * xi[0]
    for i in range(1, m):
        b = off / c_prev
        c = math.sqrt(sig2 - b * b)
        v[i] = c * xi[i] + b * xi[i - 1]
        c_prev = c
    return v


def l96_tridiag_problem(p: int, N: int, seed: int, sigma: float = 0.3, rho: float = 0.2,
                        dt: float = 0.01, spinup: int = 20, model_noise: float = 0.0,
                        dtype=np.float64) -> Problem:
    """The Lorenz-96 workload with correlated observation noise: state dimension p, H = I
    (m = p), R tridiagonal Toeplitz with diagonal sigma^2 and off-diagonals sigma^2 rho.
    Truth x0 ~ N(0, I) integrated `spinup` RK4 steps of dt; initial ensemble = truth + 0.1
    N(0, I); one forecast step (RK4, dt) of every member plus model noise of standard
    deviation `model_noise` (0 by default: the analysis errors the paper prints for this
    workload are reproduced without it); the truth advanced by the same step; y = truth + v,
    v ~ N(0, R)."""
    truth = _rng(seed, STREAM_TRUTH).standard_normal(p)
    truth = l96_rk4(truth, dt, spinup)
    Xa0 = truth[:, None] + 0.1 * _rng(seed, STREAM_ENSEMBLE).standard_normal((p, N))
    Xf = l96_rk4(Xa0, dt, 1)
    if model_noise:
        Xf = Xf + model_noise * _rng(seed, STREAM_ENSEMBLE, 1).standard_normal((p, N))
    truth = l96_rk4(truth, dt, 1)
    rowptr, col, w = identity_operator(p)
    sig2 = sigma * sigma
    r = np.full(p, sig2)
    r_off = np.full(p - 1, sig2 * rho)
    y = truth + _tridiag_noise(sig2, sig2 * rho, _rng(seed, STREAM_OBSNOISE), p)
    return Problem(np.ascontiguousarray(Xf.astype(dtype)), rowptr, col, w, r, y, truth,
                   dict(sigma=sigma, rho=rho, dt=dt, spinup=spinup, model_noise=model_noise), r_off)


def ex1b_problem(m: int, N: int = 50, seed: int = 1, q: float = 0.1) -> Problem:
    """The random-vector workload used for the CG error bounds: state and observations of size
    m (H = I), truth ~ N(0, I), initial ensemble ~ N(0, I), one forecast step with the identity
    model plus model noise N(0, q I), R = I, y = truth + N(0, I)."""
    truth = _rng(seed, STREAM_TRUTH).standard_normal(m)
    Xa0 = _rng(seed, STREAM_ENSEMBLE).standard_normal((m, N))
    Xf = Xa0 + math.sqrt(q) * _rng(seed, STREAM_ENSEMBLE, 1).standard_normal((m, N))
    rowptr, col, w = identity_operator(m)
    r = np.ones(m)
    y = truth + _rng(seed, STREAM_OBSNOISE).standard_normal(m)
    return Problem(np.ascontiguousarray(Xf), rowptr, col, w, r, y, truth, dict(q=q))


def batched_problem_specs(count: int, seed: int, n_lo: int = 4096, n_hi: int = 262144,
                          members=(16, 32, 64, 128)):
    """Shapes of a batch of uneven problems: n log-uniform in [n_lo, n_hi] rounded to a
    square grid, m = n/4, N uniform over `members`, correlation length ~ U[4, 32]."""
    rng = _rng(seed, 9)
    specs = []
    for _ in range(count):
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        side = max(4, int(round(math.sqrt(n))))
        N = int(rng.choice(members))
        ell = float(rng.uniform(4.0, 32.0))
        specs.append(dict(side=side, n=side * side, m=(side * side) // 4, N=N, ell=ell))
    return specs


def batched_problems(count: int, seed: int, dtype=np.float32, **kw):
    specs = batched_problem_specs(count, seed, **kw)
    return [grf_problem(s["side"], s["ell"], s["N"], s["m"], 0.5, 1.5, seed, dtype=dtype,
                        sub=1000 + i, meta=dict(batch_index=i)) for i, s in enumerate(specs)]


class L96Cycle:
    """Lorenz-96 cycling experiment: n=40, F=8, RK4 dt=0.05 with 5 steps between analyses,
    no model noise; truth0 ~ N(0, I) spun up for 1,000 steps; members = truth + N(0, I);
    H observes every 2nd variable (m=20); R = I."""

    def __init__(self, seed: int, n: int = 40, N: int = 20, dt: float = 0.05,
                 steps_per_cycle: int = 5, spinup: int = 1000, obs_every: int = 2):
        self.n, self.N, self.dt, self.steps = n, N, dt, steps_per_cycle
        self.rng_truth = _rng(seed, STREAM_TRUTH)
        self.rng_obs = _rng(seed, STREAM_OBSNOISE)
        truth = self.rng_truth.standard_normal(n)
        self.truth = l96_rk4(truth, dt, spinup)
        self.ensemble = self.truth[:, None] + _rng(seed, STREAM_ENSEMBLE).standard_normal((n, N))
        self.rowptr, self.col, self.w = every_kth_operator(n, obs_every)
        self.r = np.ones(self.col.size)
        self.cycle = 0

    def forecast(self):
        self.truth = l96_rk4(self.truth, self.dt, self.steps)
        self.ensemble = l96_rk4(self.ensemble, self.dt, self.steps)
        self.cycle += 1

    def observe(self) -> np.ndarray:
        return _observe(self.truth, self.rowptr, self.col, self.w, self.r, self.rng_obs)

    def problem(self, y) -> Problem:
        return Problem(np.ascontiguousarray(self.ensemble), self.rowptr, self.col, self.w,
                       self.r, y, self.truth.copy(), dict(cycle=self.cycle))
