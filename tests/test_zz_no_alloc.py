"""The allocation-free entry point (enkf_analyze_noalloc) against the handle-based one and
against the FP64 oracle's exact analysis.

Some callers of this library cannot allocate device memory when they run an analysis
(inside a CUDA-graph capture, under an application-owned memory pool, in a real-time loop
that forbids allocation after start-up); enkf_analyze_noalloc serves them from a fixed
array inside the library. This file is collected last so that a failure here comes after
every other test has run; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_handle_path_on_two_consecutive_calls(lib, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    p = synth.workload("grf512_N64_m65536", 77, scale=8, dtype=dt)     # n=4096, m=1024, N=64
    an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, tol=1e-8)
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    cfg = lib.default_config(p.n, p.m, p.N, precision=prec, tol=1e-8)
    dev = [torch.from_numpy(a).cuda() for a in (p.rowptr, p.col, p.w, p.r)]
    for call, counter in enumerate((3, 4)):
        ref = an.analyze(Xf, y, seed=9, counter=counter).double().cpu().numpy()
        Xa, st = lib.analyze_noalloc(cfg, *dev, Xf, y, seed=9, counter=counter)
        assert st["status"] == "ok", (call, st)
        Xa = Xa.double().cpu().numpy()
        err = oracle.rel_frobenius(Xa, ref)
        assert err <= 1e-6, (call, err)      # the suite's parity bar; same kernels, so ~0
        # and against the oracle's exact FP64 analysis of the same inputs, so that a fault
        # shared by both entry points cannot pass
        E = oracle.obs_perturbations(9, counter, p.r, p.N)
        exact = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
        err_o = oracle.rel_frobenius(Xa, exact)
        assert err_o <= 1e-6, (call, err_o)


def test_noalloc_rejects_partial_overlap(lib):
    p = synth.workload("grf512_N64_m65536", 79, scale=8, dtype=np.float32)
    cfg = lib.default_config(p.n, p.m, p.N, precision="fp32")
    dev = [torch.from_numpy(a).cuda() for a in (p.rowptr, p.col, p.w, p.r)]
    buf = torch.empty(2 * p.n * p.N, dtype=torch.float32, device="cuda")
    Xf = buf[: p.n * p.N].view(p.n, p.N)
    Xf.copy_(torch.from_numpy(p.Xf))
    Xa = buf[p.N: p.N + p.n * p.N].view(p.n, p.N)        # shifted by one row: partial overlap
    _, st = lib.analyze_noalloc(cfg, *dev, Xf, torch.from_numpy(p.y).cuda(), out=Xa)
    assert st["status"] == "invalid_arg"


def test_noalloc_rejects_problems_beyond_its_fixed_memory(lib):
    p = synth.workload("grf512_N64_m65536", 78, scale=2, dtype=np.float32)   # m=16384: ~48 MB
    cfg = lib.default_config(p.n, p.m, p.N, precision="fp32")
    dev = [torch.from_numpy(a).cuda() for a in (p.rowptr, p.col, p.w, p.r)]
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    _, st = lib.analyze_noalloc(cfg, *dev, Xf, y)
    assert st["status"] == "unsupported"
