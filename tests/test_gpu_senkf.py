"""GPU parity of the sEnKF comparator (Algorithm 3, Appendix A: S^{-1} replaced by the inverse
of its diagonal, X_a = X_f + X_f Z-hat^T diag(Z-hat Z-hat^T + R_N)^{-1} (Y + E - Z)) against the
oracle, on ragged shapes and the full 512^2 / N = 64 / m = 65536 workload; W is compared with
Z-hat^T diag^{-1} D built from the oracle's ensemble statistics."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_XA = {"fp64": 1e-11, "fp32": 1e-6}   # FP32 mode stores X_a in FP32 (unit roundoff 6e-8)
# W from the device's own perturbation draws: FP64 mode draws the oracle's normals exactly;
# FP32 mode evaluates Box-Muller in FP32 (each normal within ~1e-7 of the FP64 one)
TOL_W_DRAWN = {"fp64": 1e-10, "fp32": 2e-6}


def _W_ref(p, E):
    _, _, Z, _, Zhat = oracle.ensemble_stats(p.Xf.astype(np.float64), p.rowptr, p.col, p.w)
    dg = np.einsum("ij,ij->i", Zhat, Zhat) + (p.N - 1) * p.r
    return Zhat.T @ (oracle.innovations(p.y, Z, E) / dg[:, None])


def _analysis(lib, p, prec, **cfg):
    return lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, variant="senkf", **cfg)


def _dev(p, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(p.Xf)).to("cuda", dt), torch.from_numpy(p.y).cuda()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(4096, 64, 1024), (2500, 37, 999), (1600, 20, 400),
                                   (3000, 100, 700), (2048, 128, 1536), (500, 2, 130)])
def test_senkf_matches_oracle(lib, prec, shape):
    n, N, m = shape
    side = int(round(n ** 0.5))
    p = synth.grf_problem(side, 6.0, N, m, 0.5, 1.5, seed=5 * n + N + m,
                          dtype=np.float64 if prec == "fp64" else np.float32)
    an = _analysis(lib, p, prec)
    Xf, y = _dev(p, prec)
    Xa = an.analyze(Xf, y, seed=11, counter=4).double().cpu().numpy()
    st = an.stats()
    W = an.intermediates_senkf().cpu().numpy()
    E = oracle.obs_perturbations(11, 4, p.r, p.N)
    ref = oracle.senkf_alg3(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    Wr = _W_ref(p, E)
    assert st["status"] == "ok", st
    assert st["iters_max"] == 0 and st["columns_converged"] == p.N
    assert np.linalg.norm(W - Wr) <= TOL_W_DRAWN[prec] * np.linalg.norm(Wr)
    assert oracle.rel_frobenius(Xa, ref) <= TOL_XA[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_senkf_explicit_and_zero_perturbations(lib, prec):
    p = synth.workload("grf512_N64_m65536", 4, scale=8,
                       dtype=np.float64 if prec == "fp64" else np.float32)
    rng = np.random.default_rng(9)
    E = np.sqrt(p.r)[:, None] * rng.standard_normal((p.m, p.N))
    an = _analysis(lib, p, prec)
    Xf, y = _dev(p, prec)
    for Ei in (E, None):
        Ed = None if Ei is None else torch.from_numpy(Ei).cuda()
        Xa = an.analyze_with_E(Xf, y, Ed).double().cpu().numpy()
        ref = oracle.senkf_alg3(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, Ei)
        assert oracle.rel_frobenius(Xa, ref) <= TOL_XA[prec]
        W = an.intermediates_senkf().cpu().numpy()
        Wr = _W_ref(p, Ei)
        assert np.linalg.norm(W - Wr) <= 1e-10 * np.linalg.norm(Wr)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_senkf_full_size_grf512_N64_m65536(lib, prec):
    dtype = np.float64 if prec == "fp64" else np.float32
    p = synth.workload("grf512_N64_m65536", 1, dtype=dtype)
    an = _analysis(lib, p, prec)
    Xf, y = _dev(p, prec)
    Xa = an.analyze(Xf, y, seed=1, counter=0).double().cpu().numpy()
    assert an.stats()["status"] == "ok"
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    X64 = p.Xf.astype(np.float64)
    ref = oracle.senkf_alg3(X64, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, ref) <= TOL_XA[prec]
    # the comparator is an approximation: on this correlated workload it is not the EnKF
    exact = oracle.enkf_exact(X64, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, exact) > 1e-3


def test_senkf_keeps_no_m_by_N_intermediates(lib):
    p = synth.workload("grf512_N64_m65536", 2, scale=16)
    an = _analysis(lib, p, "fp64")
    Xf, y = _dev(p, "fp64")
    an.analyze(Xf, y)
    with pytest.raises(lib.EnKFError) as ei:
        an.intermediates()
    assert ei.value.status == 1


@pytest.mark.parametrize("variant", ["senkf", "reduced"])
def test_gram_variants_time_their_two_stages(lib, variant):
    # phase 0 is the Gram pass, phase 1 the N x N stage, phase 2 the update
    p = synth.workload("grf512_N64_m65536", 3, scale=4, dtype=np.float32)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", variant=variant)
    an.set_phase_timing(True)
    Xf, y = _dev(p, "fp32")
    Xa = an.analyze(Xf, y, seed=2, counter=1)
    ms = an.phase_times()
    assert all(t > 0 for t in ms), ms
    E = oracle.obs_perturbations(2, 1, p.r, p.N)
    X64 = p.Xf.astype(np.float64)
    ref = (oracle.senkf_alg3(X64, p.rowptr, p.col, p.w, p.r, p.y, E) if variant == "senkf"
           else oracle.enkf_exact(X64, p.rowptr, p.col, p.w, p.r, p.y, E))
    assert oracle.rel_frobenius(Xa.double().cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("N", [2, 37, 128])
def test_senkf_single_observation_is_the_enkf(lib, N):
    # with one observation S is 1 x 1 and equals its diagonal: Algorithm 3 is then the exact
    # EnKF analysis (Sec. 2.4's scalar gain), a property independent of the oracle's Algorithm 3
    p = synth.grf_problem(12, 3.0, N, 1, 0.5, 1.5, seed=40 + N)
    an = _analysis(lib, p, "fp64")
    Xf, y = _dev(p, "fp64")
    Xa = an.analyze(Xf, y, seed=3, counter=2).cpu().numpy()
    E = oracle.obs_perturbations(3, 2, p.r, p.N)
    exact = oracle.enkf_exact(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, exact) <= 1e-12


@pytest.mark.parametrize("variant", ["senkf", "reduced"])
@pytest.mark.parametrize("m", [1, 3, 31, 33])
@pytest.mark.parametrize("N", [2, 64, 128])
def test_gram_variants_fewer_rows_than_a_tile(lib, variant, m, N):
    # m below and around the Gram pass's 32-row tile: one CTA, ragged last tile
    p = synth.grf_problem(10, 3.0, N, m, 0.5, 1.5, seed=7 * m + N)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp64", variant=variant,
                      tol=1e-12)
    Xf, y = _dev(p, "fp64")
    Xa = an.analyze(Xf, y, seed=5, counter=1).cpu().numpy()
    assert an.stats()["status"] == "ok"
    E = oracle.obs_perturbations(5, 1, p.r, p.N)
    ref = (oracle.senkf_alg3(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E) if variant == "senkf"
           else oracle.enkf_exact(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E))
    assert oracle.rel_frobenius(Xa, ref) <= 1e-10
