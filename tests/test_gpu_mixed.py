"""GPU parity of the mixed-precision solve: BF16 / FP16 tensor-core (tcgen05) contractions
with FP32 accumulation, FP32 vectors, FP64 CG scalars, inner solves refined by an FP32
residual refresh. Bar: 1e-4 relative Frobenius error against the FP64 oracle's exact
analysis. Operands split into hi + lo parts (lowprec_terms = 3, the default) converge on
every case here; single BF16 operands only while 2 eps cond(S) stays below 1."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(lib, p, prec, seed=7, counter=3, **cfg):
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, **cfg)
    Xa = an.analyze(torch.from_numpy(np.ascontiguousarray(p.Xf, dtype=np.float32)).cuda(),
                    torch.from_numpy(p.y).cuda(), seed=seed, counter=counter)
    return an, Xa.double().cpu().numpy(), an.stats()


SHAPES = [(4096, 64, 1024), (2500, 37, 999), (1600, 20, 400), (3000, 100, 700), (2000, 97, 900),
          (20000, 128, 5000)]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("pc", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_split_mixed_matches_exact_oracle(lib, prec, pc, shape):
    n, N, m = shape
    side = int(round(n ** 0.5))
    p = synth.grf_problem(side, 6.0, N, m, 0.25, 1.0, seed=11 * n + N + m, dtype=np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-8, precondition=pc)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    err = oracle.rel_frobenius(Xa, ref)
    assert st["status"] == "ok", st
    assert err <= 1e-4, (err, st)
    # the refinement's residual is recomputed in double-float (FP64-grade) each cycle
    assert 0 < st["true_relres_max"] <= 1e-8, st


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_single_term_mixed_on_a_well_conditioned_case(lib, prec):
    p = synth.grf_problem(64, 6.0, 64, 1024, 0.25, 1.0, seed=5, dtype=np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-6, precondition=1, lowprec_terms=1)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa, ref) <= 1e-4


def test_mixed_rejects_fixed_iterations(lib):
    p = synth.workload("grf512_N64_m65536", 3, scale=16, dtype=np.float32)
    with pytest.raises(lib.EnKFError):
        lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="bf16", fixed_iters=3)


def _check_close(Xa, ref, bar, elem_bar=None):
    """The relative Frobenius error (Eq. rel_frob) within `bar` and, so that an error confined
    to one tile of a large problem cannot hide in the norm, the largest entry-wise error
    relative to the largest entry within `elem_bar` (default `bar`). The FP32 path's X_a is
    stored in FP32 and its update sums N FP32 products, so its entry-wise errors are not
    uniform: at 1024^2 / N = 128 the largest is 3.3e-6 of the largest entry while the
    Frobenius error is 5.2e-7; its entry-wise bar is ten times its Frobenius bar."""
    err = oracle.rel_frobenius(Xa, ref)
    emax = float(np.max(np.abs(Xa - ref)) / np.max(np.abs(ref)))
    eb = bar if elem_bar is None else elem_bar
    assert err <= bar and emax <= eb, (err, emax)
    return err, emax


# (N, m, grid CTAs): every CTA holds several 128-row tiles (rows per CTA = m / grid), with
# N <= 64 (double-buffered tile images) and N > 64 (NT = 128), ragged last tiles included
MULTI = [(37, 8000, 8), (64, 12000, 12), (64, 1024, 4), (100, 6000, 4), (128, 16000, 16), (128, 4100, 5)]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("pc", [0, 1])
@pytest.mark.parametrize("N,m,G", MULTI)
@pytest.mark.parametrize("order", [0, 1])
def test_split_mixed_several_tiles_per_cta(lib, prec, pc, N, m, G, order):
    # order 1: the step sums by atomic adds (N <= 64; ignored for N > 64)
    side = max(64, int(np.ceil(np.sqrt(2 * m))))
    p = synth.grf_problem(side, 6.0, N, m, 0.25, 1.0, seed=13 * m + N + G, dtype=np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-8, precondition=pc, grid_blocks=G, reduce_order=order)
    assert st["grid_blocks"] == G and (m + G - 1) // G > 128, st
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert st["status"] == "ok", st
    _check_close(Xa, ref, 1e-4)
    assert 0 < st["true_relres_max"] <= 1e-8, st


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("N,m,G", [(64, 4096, 4), (128, 4096, 8)])
def test_single_term_mixed_several_tiles_per_cta(lib, prec, N, m, G):
    # single low-precision operands on a well-conditioned case (large r), several tiles per CTA
    p = synth.grf_problem(96, 6.0, N, m, 4.0, 8.0, seed=m + N, dtype=np.float32)
    an, Xa, st = _run(lib, p, prec, tol=1e-6, precondition=1, lowprec_terms=1, grid_blocks=G)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert st["status"] == "ok", st
    _check_close(Xa, ref, 1e-4)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("order", [0, 1])
def test_full_size_grf512_N64_m65536_tensor_cores(lib, prec, order):
    """The 512 x 512 workload (n = 262,144, m = 65,536, N = 64) at full size on the automatic
    grid (several tiles per CTA), preconditioned as the benchmark runs it, with fixed-order and
    with atomic step sums. The analysis error stays at the FP32 path's level (the split
    operator and the double-float refresh): within 1e-6, the FP32 bar."""
    p = synth.workload("grf512_N64_m65536", 1, dtype=np.float32)
    an, Xa, st = _run(lib, p, prec, seed=1, counter=0, tol=1e-8, precondition=1, reduce_order=order)
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert st["status"] == "ok", st
    _check_close(Xa, ref, 1e-6, 1e-5)
    assert st["true_relres_max"] <= 1e-8, st


@pytest.fixture(scope="module")
def grf1024():
    """The mixed-precision workload at full size: 1024 x 1024 GRF (length 24), N = 128,
    m = 262,144, r ~ U[0.25, 1.0], and the oracle's exact analysis of it (N x N route)."""
    p = synth.workload("grf1024_N128_m262144", 1, dtype=np.float32)
    E = oracle.obs_perturbations(1, 0, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    return p, ref


@pytest.mark.parametrize("prec,bar,elem_bar", [("bf16", 1e-4, 1e-4), ("fp16", 1e-4, 1e-4), ("fp32", 1e-6, 1e-5)])
def test_full_size_grf1024_N128_m262144(lib, grf1024, prec, bar, elem_bar):
    p, ref = grf1024
    an, Xa, st = _run(lib, p, prec, seed=1, counter=0, tol=1e-8, precondition=1)
    assert st["status"] == "ok", st
    _check_close(Xa, ref, bar, elem_bar)
    assert st["true_relres_max"] <= 1e-8, st
    an.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("scale", [1e6, 1e-6])
@pytest.mark.parametrize("N,m,G", [(64, 1024, None), (64, 12000, 12)])
def test_split_mixed_in_any_units(lib, prec, scale, N, m, G):
    """The same problem in other units (X_f and y times s, R times s^2; the analysis scales
    by s): |HA| near 1e6 would overflow FP16 and near 1e-6 would fall into its subnormal
    range, so the tile images are scaled by a power of two chosen from the largest |HA|, and
    the Gram's z operand (R^-1 r, which scales as 1/s) by the power of two nearest the typical
    r_i. FP32 runs on the CUDA cores and needs neither."""
    side = max(64, int(np.ceil(np.sqrt(2 * m))))
    p = synth.grf_problem(side, 6.0, N, m, 0.25, 1.0, seed=29 * m + N, dtype=np.float32)
    p.Xf = (p.Xf.astype(np.float64) * scale).astype(np.float32)
    p.y = p.y * scale
    p.r = p.r * scale * scale
    extra = {} if G is None else {"grid_blocks": G}
    an, Xa, st = _run(lib, p, prec, tol=1e-8, precondition=1, reduce_order=1, **extra)
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert st["status"] == "ok", st
    _check_close(Xa, ref, 1e-4)
    assert 0 < st["true_relres_max"] <= 1e-8, st


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_nonfinite_input_ends_with_the_nonfinite_status(lib, prec):
    """A NaN in one member's state makes the ensemble mean of that element, and so a row of
    HA in every column, NaN: the refinement ends every column at its first residual refresh
    with the non-finite status (no step can make progress, so the solve stops there)."""
    q = synth.workload("grf512_N64_m65536", 15, scale=8, dtype=np.float32)
    q.Xf[q.col[3], 4] = np.nan
    an, Xa, st = _run(lib, q, prec, tol=1e-8, precondition=1)
    assert st["status"] == "nonfinite", st
    assert st["iters_max"] < 1000, st


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_identical_members(lib, prec):
    """No ensemble spread: HA = 0 and A = 0, so S = R and X_a = X_f (the images' scale is 1
    when the largest |HA| is zero)."""
    p = synth.grf_problem(64, 6.0, 16, 1024, 0.25, 1.0, seed=3, dtype=np.float32)
    p.Xf = np.repeat(p.Xf[:, :1], p.N, axis=1).copy()
    an, Xa, st = _run(lib, p, prec, tol=1e-8, precondition=1)
    assert st["status"] == "ok", st
    E = oracle.obs_perturbations(7, 3, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert np.allclose(ref, p.Xf.astype(np.float64), rtol=0, atol=1e-12 * np.abs(ref).max())
    _check_close(Xa, ref, 1e-6)
