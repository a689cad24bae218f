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
