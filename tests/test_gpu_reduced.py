"""GPU parity of CGD-EnKF-Reduced (Sec. 5.2: Algorithm 2 with CG on I + P^T P) against the
oracle: fixed CG step counts (the paper's Table 5 mode) match the oracle's iterates to
round-off; converged solves match the exact analysis; Table 5's one-step trend holds."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(lib, p, prec="fp64", seed=7, counter=3, **cfg):
    dt = torch.float64 if prec == "fp64" else torch.float32
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, variant="reduced", **cfg)
    Xa = an.analyze(torch.from_numpy(np.ascontiguousarray(p.Xf)).to("cuda", dt),
                    torch.from_numpy(p.y).cuda(), seed=seed, counter=counter)
    return an, Xa.double().cpu().numpy(), an.stats()


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_reduced_fixed_iterations_match_oracle(lib, k):
    p = synth.workload("grf512_N64_m65536", 21, scale=8)
    an, Xa, st = _run(lib, p, fixed_iters=k)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref, info = oracle.cgd_enkf_reduced(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, fixed_iters=k)
    V, G = (t.cpu().numpy() for t in an.intermediates_reduced())
    assert np.linalg.norm(G - info["G"]) <= 1e-12 * np.linalg.norm(info["G"])
    assert np.linalg.norm(V - info["V"]) <= 1e-10 * np.linalg.norm(info["V"])
    assert oracle.rel_frobenius(Xa, ref) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(4096, 64, 1024), (2500, 37, 999), (1600, 20, 400),
                                   (3000, 100, 700), (2048, 128, 1536), (500, 2, 130)])
def test_reduced_converged_matches_exact(lib, prec, shape):
    n, N, m = shape
    side = int(round(n ** 0.5))
    p = synth.grf_problem(side, 6.0, N, m, 0.5, 1.5, seed=3 * n + N + m,
                          dtype=np.float64 if prec == "fp64" else np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-12)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= (1e-9 if prec == "fp64" else 1e-6), (err, st)
    # G is N x N, so exact CG ends within N steps; at tol 1e-12 rounding costs a few more
    assert st["iters_max"] <= 3 * p.N


def test_reduced_table5_one_step_trend_on_gpu(lib):
    errs = []
    for m in (64, 1024, 16384):
        rng = np.random.default_rng(m)
        n, N = m, 20
        xt = rng.standard_normal(n)
        Xf = xt[:, None] + 0.1 * rng.standard_normal((n, N)) + 2.0
        rowptr, col, w = synth.identity_operator(n)
        r = np.full(m, 0.09)
        y = xt + 2.0 + 0.3 * rng.standard_normal(m)
        p = synth.Problem(np.ascontiguousarray(Xf), rowptr, col, w, r, y)
        an = lib.Analysis(n, m, N, rowptr, col, w, r, precision="fp64", variant="reduced",
                          fixed_iters=1, perturb_obs=0)
        Xa = an.analyze(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
        ref1, _ = oracle.cgd_enkf_reduced(Xf, rowptr, col, w, r, y, fixed_iters=1)
        assert oracle.rel_frobenius(Xa, ref1) <= 1e-10
        errs.append(oracle.rel_frobenius(Xa, oracle.enkf_alg2(Xf, rowptr, col, w, r, y)))
    assert errs[0] < errs[1] < errs[2] and errs[2] > 0.9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reduced_full_size_grf512_N64_m65536(lib, prec):
    dtype = np.float64 if prec == "fp64" else np.float32
    p = synth.workload("grf512_N64_m65536", 1, dtype=dtype)
    an, Xa, st = _run(lib, p, prec, seed=1, counter=0, tol=1e-10)
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= 1e-6, (err, st)


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("scale", [1.0, 1e-8, 1e8])
def test_reduced_fp32_double_float_gram_matches_oracle(lib, k, scale):
    """The FP32 mode forms G and the right-hand sides from FP32 ensembles with double-float
    (FP32-pair) product sums. Against the FP64 oracle on the same FP32-rounded ensemble and
    explicit FP64 perturbations, G and the fixed-k CG iterate V must agree to about 1e-11.
    Scaling X_f, y and E by s and r by s^2 leaves P = L^{-1} HA, G and V unchanged
    (Sec. 5.2), so s = 1e-8 and 1e8 (r down to 1e-16 and up to 1e16) check that the FP32
    exponent range of the pairs neither underflows nor overflows on such inputs."""
    p = synth.workload("grf512_N64_m65536", 21, scale=8, dtype=np.float32)
    Xf32 = np.ascontiguousarray((p.Xf.astype(np.float64) * scale).astype(np.float32))
    r = p.r * scale * scale
    y = p.y * scale
    E = oracle.obs_perturbations(7, 3, p.r, p.N) * scale
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, r, precision="fp32", variant="reduced",
                      fixed_iters=k)
    Xa = an.analyze_with_E(torch.from_numpy(Xf32).cuda(), torch.from_numpy(y).cuda(),
                           torch.from_numpy(E).cuda()).double().cpu().numpy()
    ref, info = oracle.cgd_enkf_reduced(Xf32.astype(np.float64), p.rowptr, p.col, p.w, r, y, E,
                                        fixed_iters=k)
    V, G = (t.cpu().numpy() for t in an.intermediates_reduced())
    assert np.linalg.norm(G - info["G"]) <= 1e-11 * np.linalg.norm(info["G"])
    assert np.linalg.norm(V - info["V"]) <= 1e-10 * np.linalg.norm(info["V"])
    # X_a itself is stored in FP32 (unit roundoff 6e-8)
    assert oracle.rel_frobenius(Xa, ref) <= 1e-6
