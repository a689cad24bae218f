"""Failure detection on the GPU without a fault: a bounded device wait that nothing releases
(a grid barrier entered by one CTA of two; an mbarrier nothing arrives on) must end at its
time limit with the timeout status, and the context must still run an analysis afterwards."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(lib, which):
    t0 = time.perf_counter()
    assert lib.selftest_wait_timeout(which, 50.0) == "timeout"
    assert time.perf_counter() - t0 < 5.0               # ended at its limit, not at 4 s or never
    # the same context still runs an analysis that matches the oracle
    p = synth.workload("grf512_N64_m65536", 4, scale=8, dtype=np.float32)
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", tol=1e-8)
    E = oracle.obs_perturbations(3, 0, p.r, p.N)
    Xa = an.analyze_with_E(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(p.y).cuda(),
                           torch.from_numpy(E).cuda())
    assert an.stats()["status"] == "ok"
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    assert oracle.rel_frobenius(Xa.double().cpu().numpy(), ref) <= 1e-6
    an.close()
