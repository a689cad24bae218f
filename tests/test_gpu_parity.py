"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element,
on seeded inputs. Bars: rel. Frobenius error (Eq. rel_frob) against the exact analysis
<= 1e-6 for the FP64 and FP32 paths; fixed-iteration FP64 CG iterates equal to the oracle's
up to round-off (1e-11); perturbations within 1e-14 relative (the integer Philox stream is
identical; log/sincos may differ in the last bits)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _csr_problem(n, N, m, seed, dtype=np.float64):
    """Random general CSR operator (1..3 weighted entries per row), non-uniform R."""
    rng = np.random.default_rng(seed)
    Xf = (rng.standard_normal((n, N)) + 2.0 * rng.standard_normal(n)[:, None]).astype(dtype)
    rowptr, col, w = [0], [], []
    for _ in range(m):
        k = int(rng.integers(1, 4))
        col += list(rng.choice(n, size=k, replace=False))
        w += list(rng.uniform(-1.5, 1.5, size=k))
        rowptr.append(len(col))
    r = rng.uniform(0.3, 2.0, size=m)
    y = rng.standard_normal(m) * 2.0
    return synth.Problem(np.ascontiguousarray(Xf), np.array(rowptr, np.int32),
                         np.array(col, np.int32), np.array(w), r, y)


def _run(lib, p, prec="fp64", seed=7, counter=3, E=None, **cfg):
    dt = torch.float64 if prec == "fp64" else torch.float32
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, **cfg)
    Xf = torch.from_numpy(np.ascontiguousarray(p.Xf)).to("cuda", dt)
    y = torch.from_numpy(p.y).to("cuda", torch.float64)
    if E is None:
        Xa = an.analyze(Xf, y, seed=seed, counter=counter)
    else:
        Xa = an.analyze_with_E(Xf, y, None if E is False else torch.from_numpy(E).cuda())
    st = an.stats()
    return an, Xa.double().cpu().numpy(), st


def _oracle_exact(p, E):
    return oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)


def test_perturbations_match_oracle_generator(lib):
    r = np.random.default_rng(0).uniform(0.2, 3.0, size=3001)
    for N, seed, counter in ((64, 7, 3), (37, 2 ** 40 + 5, 2 ** 33 + 1), (2, 0, 0)):
        E = lib.draw_perturbations(seed, counter, torch.from_numpy(r).cuda(), N).cpu().numpy()
        ref = oracle.obs_perturbations(seed, counter, r, N)
        assert np.max(np.abs(E - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_single_precision_perturbations_in_fp32_mode(lib):
    # The FP32 and tensor-core modes draw the Box-Muller normals in FP32 from the same Philox
    # uniforms; the innovations D = y + E - H X_f they form must agree with the oracle's (E
    # drawn in FP64) to about 1e-7 of the perturbation scale, tails included (m N / 2 = 640 k
    # pairs reach uniforms within 1e-5 of 0 and of 1).
    p = synth.workload("grf512_N64_m65536", 21, scale=2, dtype=np.float32)   # n = 65,536, m = 16,384, N = 64
    for prec in ("fp32", "fp16"):
        an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, tol=1e-8,
                          precondition=1)
        Xf = torch.from_numpy(p.Xf).cuda()
        an.analyze(Xf, torch.from_numpy(p.y).cuda(), seed=9, counter=4)
        _, D, _, _ = (t.cpu().numpy() for t in an.intermediates())
        E = oracle.obs_perturbations(9, 4, p.r, p.N)
        Dref = oracle.innovations(p.y, oracle.apply_H(p.rowptr, p.col, p.w, p.Xf.astype(np.float64)), E)
        err = np.abs(D - Dref) / np.sqrt(p.r)[:, None]
        assert err.max() <= 2e-6, (prec, err.max())
        assert np.sqrt(np.mean(err ** 2)) <= 2e-7, (prec, np.sqrt(np.mean(err ** 2)))
        an.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(4096, 64, 1024), (2500, 37, 999), (1600, 20, 400),
                                   (3000, 100, 700), (2048, 128, 1536), (500, 2, 130)])
def test_analysis_matches_exact_oracle(lib, prec, shape):
    n, N, m = shape
    side = int(round(n ** 0.5))
    p = synth.grf_problem(side, 6.0, N, m, 0.5, 1.5, seed=n + N + m,
                          dtype=np.float64 if prec == "fp64" else np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-10)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = _oracle_exact(p, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= 1e-6, (err, st)
    if prec == "fp64":
        assert err <= 1e-8, (err, st)
        assert st["true_relres_max"] <= 1e-9


def test_general_csr_operator_and_explicit_E(lib):
    p = _csr_problem(900, 24, 333, 5)
    E = np.random.default_rng(9).standard_normal((p.m, p.N)) * np.sqrt(p.r)[:, None]
    an, Xa, st = _run(lib, p, "fp64", E=E, tol=1e-12)
    ref = oracle.enkf_alg1(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, ref) <= 1e-9
    # E = NULL is the paper's unperturbed EnKF
    an, Xa0, st = _run(lib, p, "fp64", E=False, tol=1e-12)
    ref0 = oracle.enkf_alg1(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, None)
    assert oracle.rel_frobenius(Xa0, ref0) <= 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 5, 12])
def test_fixed_iteration_cg_iterates_match_oracle(lib, k):
    p = synth.workload("grf512_N64_m65536", 11, scale=8)
    an, Xa, st = _run(lib, p, "fp64", fixed_iters=k)
    HA, D, Z, W = (t.cpu().numpy() for t in an.intermediates())
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    Xa_ref, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, fixed_iters=k)
    assert np.linalg.norm(HA - info["Zhat"]) <= 1e-13 * np.linalg.norm(info["Zhat"])
    assert np.linalg.norm(D - info["D"]) <= 1e-13 * np.linalg.norm(info["D"])
    assert np.linalg.norm(Z - info["Z"]) <= 1e-11 * np.linalg.norm(info["Z"])
    assert np.linalg.norm(W - info["W"]) <= 1e-11 * np.linalg.norm(info["W"])
    assert oracle.rel_frobenius(Xa, Xa_ref) <= 1e-11
    it, _, _ = an.column_stats()
    assert np.all(it == k)


def test_iteration_counts_match_oracle_stopping_rule(lib):
    p = synth.workload("grf512_N64_m65536", 12, scale=8)
    an, Xa, st = _run(lib, p, "fp64", tol=1e-8)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    _, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E, tol=1e-8)
    it, rel, _ = an.column_stats()
    # FP64 rounding differs between the two implementations; near the tolerance a column
    # can need a few more or fewer steps, so most columns must agree exactly and all closely
    diff = np.abs(it - info["iters"])
    assert np.mean(diff == 0) >= 0.75 and diff.max() <= max(3, int(0.06 * info["iters"].max()))
    assert np.all(rel <= 1e-8)


def test_lemma1_equal_variances_converge_within_N_plus_1(lib):
    p = synth.workload("grf512_N64_m65536", 13, scale=8)
    p.r[:] = 0.8
    an, Xa, st = _run(lib, p, "fp64", tol=1e-12, max_iter=p.N + 1)
    assert st["status"] == "ok" and st["iters_max"] <= p.N + 1


def test_in_place_and_host_api_and_determinism(lib):
    p = synth.workload("grf512_N64_m65536", 14, scale=8, dtype=np.float32)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32")
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    a = an.analyze(Xf, y, seed=1, counter=2)
    b = an.analyze(Xf, y, seed=1, counter=2)
    assert torch.equal(a, b)                       # fixed-order reductions: bitwise repeatable
    Xh = torch.from_numpy(p.Xf).pin_memory()
    c = an.analyze_host(Xh, torch.from_numpy(p.y).pin_memory(), seed=1, counter=2)
    assert torch.equal(a.cpu(), c)
    X2 = Xf.clone()
    an.analyze(X2, y, seed=1, counter=2, out=X2)   # in place
    assert torch.equal(a, X2)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16"])
def test_host_api_pinned_and_pageable_buffers(lib, prec):
    """enkf_analyze_host: pinned X_f (innovations read host memory while X_f uploads on a second
    stream), pinned or pageable X_a, pageable inputs (staged copies), in place on a pinned
    buffer, and twice in a row on one handle: every combination equals enkf_analyze bitwise."""
    dt = np.float64 if prec == "fp64" else np.float32
    p = synth.workload("grf512_N64_m65536", 16, scale=4, dtype=dt)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec)
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    ref = an.analyze(Xf, y, seed=3, counter=4).cpu()
    yp = torch.from_numpy(p.y).pin_memory()
    for pin_in in (True, False):
        for pin_out in (True, False):
            Xh = torch.from_numpy(p.Xf.copy())
            Xh = Xh.pin_memory() if pin_in else Xh
            out = torch.empty(tuple(Xh.shape), dtype=Xh.dtype, pin_memory=pin_out)
            for _ in range(2):
                c = an.analyze_host(Xh, yp if pin_in else torch.from_numpy(p.y), seed=3, counter=4, out=out)
                assert torch.equal(c, ref), (pin_in, pin_out)
            assert torch.equal(Xh, torch.from_numpy(p.Xf))   # the input is left as it was
    Xh = torch.from_numpy(p.Xf.copy()).pin_memory()
    an.analyze_host(Xh, yp, seed=3, counter=4, out=Xh)      # in place on a pinned buffer
    assert torch.equal(Xh, ref)


def test_zero_innovation_column_and_tiny_problem(lib):
    p = _csr_problem(40, 20, 20, 21)
    Z = oracle.apply_H(p.rowptr, p.col, p.w, p.Xf)
    E = np.random.default_rng(3).standard_normal((p.m, p.N))
    E[:, 5] = Z[:, 5] - p.y                        # d_5 = 0 exactly
    an, Xa, st = _run(lib, p, "fp64", E=E, tol=1e-12)
    ref = oracle.enkf_alg1(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, ref) <= 1e-10
    it, rel, _ = an.column_stats()
    assert it[5] == 0


def test_not_converged_and_nonfinite_statuses(lib):
    p = synth.workload("grf512_N64_m65536", 15, scale=8)
    an, Xa, st = _run(lib, p, "fp64", tol=1e-12, max_iter=3)
    assert st["status"] == "not_converged" and np.all(np.isfinite(Xa))
    q = synth.workload("grf512_N64_m65536", 15, scale=8)
    q.Xf[q.col[3], 4] = np.nan
    an, Xa, st = _run(lib, q, "fp64", tol=1e-8)
    assert st["status"] == "nonfinite"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_grf512_N64_m65536(lib, prec):
    """The benchmark workload at full size (n=262,144, m=65,536, N=64, tol 1e-8), in the
    launch configuration bench.py times, against the exact oracle (N x N route)."""
    dtype = np.float64 if prec == "fp64" else np.float32
    p = synth.workload("grf512_N64_m65536", 1, dtype=dtype)
    an, Xa, st = _run(lib, p, prec, seed=1, counter=0, tol=1e-8)
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    ref = _oracle_exact(p, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= 1e-6, (err, st)
    assert st["true_relres_max"] <= 1e-8


def test_l96_cycling_lockstep(lib):
    """Lorenz-96 (n=40, N=20, m=20, R=I, tol 1e-10): 200 cycles in lockstep. Every cycle the
    GPU and the oracle analyse the same forecast ensemble with the same perturbations, and
    the oracle's analysis is propagated (the chaotic model amplifies last-bit differences,
    so a GPU-driven trajectory would separate from the oracle's after a few dozen cycles)."""
    cyc = synth.L96Cycle(seed=4)
    an = lib.Analysis(40, cyc.col.size, 20, cyc.rowptr, cyc.col, cyc.w, cyc.r, precision="fp64",
                      tol=1e-10)
    for k in range(200):
        cyc.forecast()
        y = cyc.observe()
        Xa = an.analyze(torch.from_numpy(cyc.ensemble).cuda(), torch.from_numpy(y).cuda(),
                        seed=99, counter=k).cpu().numpy()
        assert an.stats()["status"] == "ok"
        E = oracle.obs_perturbations(99, k, cyc.r, 20)
        ref = oracle.enkf_alg1(cyc.ensemble, cyc.rowptr, cyc.col, cyc.w, cyc.r, y, E)
        err = oracle.rel_frobenius(Xa, ref)
        assert err <= 1e-8, (k, err)
        cyc.ensemble = ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(4096, 64, 1024), (2500, 37, 999), (1600, 20, 400),
                                   (3000, 100, 700), (500, 2, 130)])
def test_preconditioned_cg_matches_exact_oracle(lib, prec, shape):
    """CG preconditioned by R (Jacobi) converges to the same analysis; R^-1/2 S R^-1/2 is the
    identity plus a rank < N term, so exact CG would end within N steps; with r spread over
    [0.05, 5] rounding adds some (bounded here by 2N in FP64)."""
    n, N, m = shape
    side = int(round(n ** 0.5))
    p = synth.grf_problem(side, 6.0, N, m, 0.05, 5.0, seed=7 * n + N + m,
                          dtype=np.float64 if prec == "fp64" else np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-10, precondition=1)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = _oracle_exact(p, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= (1e-8 if prec == "fp64" else 1e-6), (err, st)
    if prec == "fp64":
        assert st["iters_max"] <= 2 * p.N, st
    an0, Xa0, st0 = _run(lib, p, prec, tol=1e-10, precondition=0)
    assert st0["iters_max"] >= st["iters_max"]


@pytest.mark.parametrize("order", [0, 1])
def test_preconditioned_full_size_grf512_N64_m65536_fp32(lib, order):
    p = synth.workload("grf512_N64_m65536", 1, dtype=np.float32)
    an, Xa, st = _run(lib, p, "fp32", seed=1, counter=0, tol=1e-8, precondition=1, reduce_order=order)
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    err = oracle.rel_frobenius(Xa, _oracle_exact(p, E))
    assert st["status"] == "ok" and err <= 1e-6, (err, st)


@pytest.mark.parametrize("N,m,G,pc", [(37, 3000, 6, 1), (64, 5000, 9, 0), (100, 4000, 7, 1), (128, 6000, 11, 1)])
def test_fp32_atomic_step_sums_match_oracle(lib, N, m, G, pc):
    """reduce_order = 1 in the FP32 mode: each step's Gram and column sums are added into
    rotating accumulators by atomic adds (one grid barrier per step; N > 64 keeps the
    fixed-order reduction); ragged N (N % 4 != 0), plain and preconditioned CG, several CTAs,
    against the exact analysis."""
    p = _csr_problem(2 * m, N, m, 100 + N, dtype=np.float32)
    E = np.random.default_rng(N).standard_normal((m, N)) * np.sqrt(p.r)[:, None]
    an, Xa, st = _run(lib, p, "fp32", E=E, tol=1e-8, precondition=pc, grid_blocks=G, reduce_order=1)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok" and err <= 1e-6, (err, st)
    assert st["grid_blocks"] == G


def test_fp32_intermediates_are_the_double_float_arrays(lib):
    # In the FP32 mode HA and Z exist only as FP32 pairs; the intermediates widen them: HA to
    # about 48 bits of the oracle's, Z to the solution within the analysis tolerance, and
    # W = HA^T Z / (N - 1) consistent with both.
    p = synth.workload("grf512_N64_m65536", 5, scale=4, dtype=np.float32)   # m = 4,096, N = 64
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", tol=1e-9,
                      precondition=1)
    E = oracle.obs_perturbations(8, 1, p.r, p.N)
    an.analyze_with_E(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(p.y).cuda(), torch.from_numpy(E).cuda())
    assert an.stats()["status"] == "ok"
    HA, D, Z, W = (t.cpu().numpy() for t in an.intermediates())
    Xf = p.Xf.astype(np.float64)
    _, _, _, _, HAref = oracle.ensemble_stats(Xf, p.rowptr, p.col, p.w)
    assert np.max(np.abs(HA - HAref)) <= 1e-13 * np.max(np.abs(HAref))
    S_Z = oracle.S_matvec(HAref, p.r, Z)
    assert np.linalg.norm(S_Z - D) <= 1e-9 * np.linalg.norm(D)         # the stopping rule, tol 1e-9
    assert np.max(np.abs(W - HA.T @ Z / (p.N - 1))) <= 1e-10 * np.max(np.abs(W))
    an.close()
