"""GPU parity of the learned warm start against the FP64 oracle (oracle/warmstart.py): MLP
forward, loss gradient (the gradient check), Adam, standardisation, the training-pair
features and targets of an analysis, and the warm-started analysis itself (whose result
must still match the exact analysis, whatever the model predicts)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import warmstart as ows
from synth.mlp_init import init_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(37, 50, 2, 13, 70), (1088, 512, 3, 64, 64), (130, 64, 1, 16, 129)]


def _params(shape, seed):
    p = init_params(*shape, seed=seed, out_scale=1.0)
    rng = np.random.default_rng(seed)
    n_in, n_out = shape[0], shape[3]
    P = p.size
    p[P - 2 * n_in - 2 * n_out:P - n_in - 2 * n_out] = rng.standard_normal(n_in) * 0.3          # mu_in
    p[P - n_in - 2 * n_out:P - 2 * n_out] = rng.uniform(0.5, 2.0, n_in)                        # sd_in
    p[P - 2 * n_out:P - n_out] = rng.standard_normal(n_out) * 0.3                              # mu_out
    p[P - n_out:] = rng.uniform(0.5, 2.0, n_out)                                               # sd_out
    return p


@pytest.mark.parametrize("dims", SHAPES)
def test_mlp_forward_matches_oracle(lib, dims):
    shape, B = dims[:4], dims[4]
    p = _params(shape, 1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((B + 5, shape[0])).astype(np.float32)
    rows = rng.permutation(B + 5)[:B].astype(np.int32)
    Y = lib.mlp_forward(shape, torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(),
                        torch.from_numpy(rows).cuda()).cpu().numpy()
    ref = ows.forward(p.astype(np.float64), shape, X[rows].astype(np.float64))
    assert np.max(np.abs(Y - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("dims", SHAPES)
def test_mlp_gradient_matches_oracle(lib, dims):
    shape, B = dims[:4], dims[4]
    p = _params(shape, 3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((B, shape[0])).astype(np.float32)
    T = rng.standard_normal((B, shape[3])).astype(np.float32)
    loss, grad = lib.mlp_loss_grad(shape, torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(),
                                   torch.from_numpy(T).cuda())
    L, g = ows.loss_grad(p.astype(np.float64), shape, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    gg = grad.cpu().numpy()[:g.size]
    trained = lib.mlp_trained_count(shape)
    # per layer, elementwise within 1e-4 of that layer's largest gradient entry
    off = 0
    for fi, fo in ows.layer_dims(*shape):
        for cnt in (fi * fo, fo):
            a, b = gg[off:off + cnt], g[off:off + cnt]
            assert np.max(np.abs(a - b)) <= 1e-4 * max(np.max(np.abs(b)), 1e-30), (fi, fo, cnt)
            off += cnt
    assert off == trained


def test_adam_matches_oracle(lib):
    rng = np.random.default_rng(5)
    n = 10007
    theta = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    tp, tm, tv = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (theta, m, v))
    for step in range(1, 6):
        g = rng.standard_normal(n)
        lib.mlp_adam(n, tp, torch.from_numpy(g.astype(np.float32)).cuda(), tm, tv, step, 1e-2)
        theta, m, v = ows.adam(theta, g.astype(np.float32).astype(np.float64), m, v, step, 1e-2)
    assert np.max(np.abs(tp.cpu().numpy() - theta)) <= 1e-5


def test_standardize_matches_oracle(lib):
    shape = (20, 8, 1, 5)
    rng = np.random.default_rng(6)
    X = (rng.standard_normal((3001, 20)) * rng.uniform(0.1, 3, 20) + rng.standard_normal(20)).astype(np.float32)
    X[:, 3] = 2.5   # constant feature -> sd 1
    T = rng.standard_normal((3001, 5)).astype(np.float32)
    p = torch.from_numpy(init_params(*shape, seed=0)).cuda()
    lib.mlp_standardize(shape, p, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    _, mu_in, sd_in, mu_out, sd_out = ows.unpack(p.cpu().numpy(), *shape)
    rmx, rsx, rmt, rst = ows.standardization(X, T)
    for a, b in ((mu_in, rmx), (sd_in, rsx), (mu_out, rmt), (sd_out, rst)):
        assert np.max(np.abs(a - b)) <= 1e-5 * max(1.0, np.max(np.abs(b)))
    assert sd_in[3] == 1.0


def _grf_small(seed, N=16, side=40):
    return synth.grf_problem(side, 6.0, N, (side * side) // 4, 0.5, 1.5, seed, dtype=np.float32, sub=seed)


def test_features_and_targets_match_oracle(lib):
    p = _grf_small(7)
    K = 64
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1)
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    an.analyze(Xf, y, seed=3, counter=1)
    F, T = an.warm_features(K)
    E = oracle.obs_perturbations(3, 1, p.r, p.N)
    _, info = oracle.cgd_enkf(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E, tol=1e-13)
    HA, D, Z = info["Zhat"], info["D"], info["Z"]
    Fr, s = ows.features(HA, D, p.r, K)
    W = HA.T @ Z / (p.N - 1)
    Tr = ows.targets(W, s)
    assert np.max(np.abs(F.cpu().numpy() - Fr)) <= 1e-5 * np.max(np.abs(Fr))
    assert np.max(np.abs(T.cpu().numpy() - Tr)) <= 1e-5 * np.max(np.abs(Tr))


@pytest.mark.parametrize("scale,expect_fallback,accept", [(1.0, False, 0), (1e8, True, 0), (1.0, False, 1)])
def test_warm_started_analysis_matches_exact(lib, scale, expect_fallback, accept):
    p = _grf_small(9)
    K = 64
    shape = (K + p.N, 64, 2, p.N, 0)[:4]
    params = init_params(*shape, seed=1, out_scale=1.0)
    nw = lib.mlp_trained_count(shape)
    params[:nw] *= scale ** (1.0 / 3.0)   # scale ** 1 over the three layers: a wild model
    pt = torch.from_numpy(params).cuda()
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1, warm_start=1,
                      warm_accept=accept)
    an.set_warm_model(shape, pt)
    Xa = an.analyze(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(p.y).cuda(), seed=5, counter=0)
    st = an.stats()
    assert st["status"] == "ok"
    assert st["warm_relres_max"] >= 0.0
    if expect_fallback:
        assert st["warm_fallbacks"] == p.N
    if accept:
        assert st["warm_fallbacks"] == 0   # every finite start is kept
    E = oracle.obs_perturbations(5, 0, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa.double().cpu().numpy(), ref) <= 1e-6


def test_warm_start_requires_model(lib):
    p = _grf_small(10)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", warm_start=1)
    with pytest.raises(lib.EnKFError, match="no model"):
        an.analyze(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(p.y).cuda())
    with pytest.raises(lib.EnKFError):
        lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp64", warm_start=1)


def test_trained_model_gain(lib):
    """Train on pairs from the method's own solves (small GRF case) with the library's
    kernels, then compare CG iterations from the learned start and from zero on held-out
    seeds. The analysis must stay exact either way; the gain is reported."""
    from paper_2606_19224_gb300 import warm_train as wt
    res, _ = wt.run(dict(wt.SMALL), log=lambda *_: None)
    print("learned warm start:", {k: res[k] for k in ("pairs", "loss_first", "loss_last", "iters_mean_zero",
                                                       "iters_mean_learned", "iters_mean_learned_accept",
                                                       "ms_zero", "ms_learned", "ms_learned_accept")})
    assert res["loss_last"] < 0.5 * res["loss_first"]
    for r in res["eval"]:
        for mode in ("zero", "learned", "learned_accept"):
            assert r[mode]["status"] == "ok"
        assert r["rel_diff_zero_vs_learned"] <= 2e-6
        assert r["rel_diff_zero_vs_learned_accept"] <= 2e-6
    assert res["iters_mean_learned"] <= res["iters_mean_zero"]
