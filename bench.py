#!/usr/bin/env python3
"""Benchmark of the CGD-EnKF analysis step on GB300.

One step = one full analysis (observation gather + anomalies + perturbed innovations, the
persistent CG solve of S Z = D, and the ensemble update X_a = X_f + A W) through the C ABI
on the synthetic 512x512 Gaussian-random-field workload: n = 262,144 state variables,
N = 64 members, m = 65,536 randomly placed observations, r ~ U[0.5, 1.5], CG tolerance
1e-8 (true FP64 relative residual).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). `value` is analyses/s summed over ranks (each rank runs its
own independent analyses: weak scaling, no collective on the data path). The headline path
is the FP32 CG with FP64 residual refresh (meets 1e-6 relative Frobenius error); the plain
FP64 GPU CG is timed beside it. `--impl reference` times the CPU oracle instead (host cores).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "grf512_N64_m65536"
METRIC = "analysis steps/s and HBM-roofline fraction vs plain FP64 GPU CG at stated error"
UNIT = "analyses/s"
L2_FLUSH_BYTES = 256 << 20
BATCH_WORKLOAD = "batched256_grf"
MIXED_WORKLOAD = "grf1024_N128_m262144"


def B_ITER(m, N):
    """Algorithmic DRAM bytes of one fused FP32 CG step (Chronopoulos-Gear form): HA read
    once (4 m N), the iterate, residual, direction and S-direction read and written
    (4 x 8 m N), r read (4 m)."""
    return 36 * m * N + 4 * m


def B_REF(m, N):
    """Algorithmic DRAM bytes of one double-float residual refresh: pass A reads HA (8 m N),
    reads and writes Z (16 m N) and reads X (4 m N); pass B reads HA, Z and D (24 m N) and
    writes the next right-hand side (4 m N)."""
    return 56 * m * N

# DRAM bytes (read + write) of one solve launch on this workload per precision, from the ncu
# captures summarised in profiles/solve_kernel_fp32_grf512_N64_m65536.md and
# profiles/solve_mixed_kernel_fp16_grf512_N64_m65536.md, with the hash of the kernel sources
# each capture measured; reported as null once those sources have changed.
NCU_TRAFFIC = {"fp32": {"bytes": 4.646017e9, "src_sha": "f359344179649ea3"},
               "fp16": {"bytes": 6.431757e9, "src_sha": "18d941411bdfab5b"}}
# The same for one batch_kernel launch on the 256-problem batch (seed 1), from the one-pass
# DRAM capture summarised in profiles/batch_kernel_batched256_grf_dram.md.
NCU_TRAFFIC_BATCH = {"bytes": 1.436453e12, "problems": 256, "seed": 1, "src_sha": "869cf69968486ece"}
_KERNEL_SOURCES = {
    "fp32": ("kernels_fp.cu", "common.cuh", "cg_device.cuh", "solve_body.cuh"),
    "fp16": ("kernels_tc.cu", "kernels_tc_fp16.cu", "tc_mixed.cuh", "common.cuh", "cg_device.cuh"),
    "bf16": ("kernels_tc.cu", "kernels_tc_bf16.cu", "tc_mixed.cuh", "common.cuh", "cg_device.cuh"),
    "batch": ("kernels_batch.cu", "solve_body.cuh", "innov_device.cuh", "common.cuh", "cg_device.cuh"),
}


def _src_hash(precision="fp32"):
    h = hashlib.sha256()
    for f in _KERNEL_SOURCES[precision]:
        with open(os.path.join(ROOT, "paper_2606_19224_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# FP32 instruction rate of a GB300 at its 2.07 GHz maximum clock: 152 SMs x 128 FP32 lanes,
# one operation per lane and clock (tera-operations per second)
FP32_OPS_PEAK_T = 152 * 128 * 2.07e9 / 1e12
# FP32 operations per term of a double-float product sum (exact product by FMA with the
# cross terms, TwoSum into the running sum, error gathered in the compensation word)
DF_OPS_PER_TERM = 12


def _gram_roofline(terms, ms):
    """The Gram pass of the Reduced and sEnKF variants on an FP32 ensemble: double-float
    product sums, bound by the FP32 issue rate (`terms` products per launch)."""
    ops = DF_OPS_PER_TERM * terms
    achieved = ops / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_OPS_PEAK_T, "unit": "T FP32 op/s",
            "frac": achieved / FP32_OPS_PEAK_T, "ops_per_launch": ops, "terms_per_launch": terms,
            "launch_ms": ms, "peak_source": "FP32 lanes x maximum SM clock"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _rank_seed(seed, rank):
    """Each rank analyses its own seeded problems (weak scaling): seeds 1000 apart."""
    return seed + 1000 * rank


def _max_over_ranks(x, dev, ws):
    """The slowest rank's figure (the job's time): all_reduce MAX of one float64 on `dev`."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank, seconds, ws):
    """Whole-job throughput: the units all ws ranks processed over the slowest rank's time."""
    return ws * units_per_rank / seconds


def _cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info()), default=0)
        if n:
            return n
    except Exception:
        pass
    return len(os.sched_getaffinity(0))


def cpu_baseline(problem, E, budget_s=20.0):
    """The CPU oracle as it stands on the host cores: exact analysis through Algorithm 2
    (N x N Cholesky), repeated on the benchmark's full-size problem within the budget."""
    import oracle
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.enkf_exact(problem.Xf.astype("float64"), problem.rowptr, problem.col, problem.w,
                          problem.r, problem.y, E)
        reps += 1
        el = time.perf_counter() - t0
        if el > budget_s or reps >= 8:
            break
    return {"value": reps / el, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{reps} full-size exact analyses ({WORKLOAD}, Algorithm 2 route, FP64 numpy) "
                      f"in {el:.1f} s"}


def cpu_baseline_one_core(seed, reps=3):
    """The same oracle on one thread (BLAS and OpenMP limited to 1), in a child process so that
    the limit holds from its first import; the analyses are the benchmark's full-size problem."""
    import subprocess
    import sys
    code = ("import time\nimport numpy as np\nimport oracle, synth\n"
            f"p = synth.workload({WORKLOAD!r}, {int(seed)}, dtype=np.float32)\n"
            f"E = oracle.obs_perturbations({int(seed)}, 0, p.r, p.N)\n"
            "X = p.Xf.astype('float64')\n"
            "t0 = time.perf_counter()\n"
            f"for _ in range({int(reps)}):\n"
            "    oracle.enkf_exact(X, p.rowptr, p.col, p.w, p.r, p.y, E)\n"
            "print(time.perf_counter() - t0)\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900, check=True)
    el = float(out.stdout.strip().splitlines()[-1])
    return {"value": reps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} full-size exact analyses ({WORKLOAD}, Algorithm 2 route, FP64 numpy) "
                      f"on one thread in {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    p = synth.workload(WORKLOAD, args.seed, dtype=np.float32)
    E = oracle.obs_perturbations(args.seed, 0, p.r, p.N)
    for _ in range(args.warmup):
        oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    t0 = time.perf_counter()
    for k in range(args.steps):
        E = oracle.obs_perturbations(args.seed, k, p.r, p.N)
        oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": p.n, "m": p.m, "N": p.N, "tol": 1e-8,
                       "route": "CPU oracle, exact FP64 analysis (Algorithm 2, N x N Cholesky)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                             "sample": f"{args.steps} full-size exact analyses, perturbations "
                                       f"from the oracle's Philox stream"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2606_19224_gb300 as enkf
    import synth

    seed = _rank_seed(args.seed, rank)
    p = synth.workload(WORKLOAD, seed, dtype=np.float32)
    n, m, N = p.n, p.m, p.N
    an = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision=args.precision, tol=1e-8,
                       precondition=args.precondition)
    an.set_phase_timing(True)
    Xf = torch.from_numpy(p.Xf).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    out = torch.empty_like(Xf)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for k in range(args.warmup):
        an.analyze(Xf, y, seed, k, out=out)
    st = an.stats()
    if st["status"] != "ok":
        raise SystemExit(f"warm-up analysis failed: {st}")

    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    solve_ms, iters, refines = [], [], []
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))                      # L2 flush, outside the timed window
        ev[k][0].record(stream)
        an.analyze(Xf, y, seed, args.warmup + k, out=out)
        ev[k][1].record(stream)
        ph = an.phase_times()                      # syncs on the last kernel's event
        solve_ms.append(ph[1])
        s = an.stats()
        iters.append(s["iters_max"])
        refines.append(s["refinements"])
    barrier()
    clk = clocks.stop()
    ms = _max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev, ws)
    value = _job_rate(args.steps, ms / 1e3, ws)
    last_status = an.stats()

    # end to end through the host-buffer entry point (pinned host memory, copies inside)
    Xh = torch.from_numpy(p.Xf).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    Xo = torch.empty_like(Xh).pin_memory()
    for k in range(2):
        an.analyze_host(Xh, yh, seed, k, out=Xo)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 4)
    for k in range(e2e_steps):
        an.analyze_host(Xh, yh, seed, k, out=Xo)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dev, ws)
    e2e = {"value": _job_rate(e2e_steps, e2e_s, ws), "unit": UNIT,
           "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 8),
           "d2h_bytes_per_step": int(Xo.numel() * 4)}

    # the same FP32 path with plain (unpreconditioned) CG, for reference
    an_plain = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision="fp32", tol=1e-8,
                             precondition=0)
    an_plain.analyze(Xf, y, seed, 0, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.fp64_steps):
        an_plain.analyze(Xf, y, seed, k, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    plain32_ms = e0.elapsed_time(e1) / args.fp64_steps
    s_plain = an_plain.stats()
    an_plain.close()

    # plain FP64 GPU CG on the same problem (the comparison point)
    p64 = synth.workload(WORKLOAD, seed, dtype=np.float64)
    an64 = enkf.Analysis(n, m, N, p64.rowptr, p64.col, p64.w, p64.r, precision="fp64", tol=1e-8)
    X64 = torch.from_numpy(p64.Xf).to(dev)
    o64 = torch.empty_like(X64)
    an64.analyze(X64, y, seed, 0, out=o64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.fp64_steps):
        an64.analyze(X64, y, seed, k, out=o64)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1) / args.fp64_steps
    s64 = an64.stats()
    an64.set_phase_timing(True)                    # the solve kernel alone, for the context leg
    an64.analyze(X64, y, seed, 0, out=o64)
    fp64_solve_ms = float(an64.phase_times()[1])
    an64.set_phase_timing(False)

    # the two variants built on one Gram pass over the observation rows, on the same FP32
    # ensemble, L2 flushed before each timed analysis: CGD-EnKF-Reduced (Algorithm 2 with CG on
    # the N x N system) and the paper's sEnKF comparator (Algorithm 3: S^{-1} replaced by its
    # diagonal's inverse, no solve); phases = (Gram pass, N x N stage, update)
    def time_variant(an_v):
        an_v.set_phase_timing(True)
        an_v.analyze(Xf, y, seed, 0, out=out)
        tot, ph = [], []
        for k in range(max(3, args.fp64_steps)):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            an_v.analyze(Xf, y, seed, k, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            tot.append(e0.elapsed_time(e1))
            ph.append(an_v.phase_times())
        return float(np.mean(tot)), [float(v) for v in np.mean(np.array(ph), axis=0)]

    an_r = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision="fp32", variant="reduced", tol=1e-8)
    reduced_ms, reduced_ph = time_variant(an_r)
    reduced_st = an_r.stats()
    an_s = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision="fp32", variant="senkf")
    senkf_ms, senkf_ph = time_variant(an_s)

    if rank != 0:
        return
    # context only, so that the FP64 comparison point is visibly not a strawman: the same plain
    # FP64 CG written with PyTorch (cuBLAS DGEMM for the two contractions of every matvec, a
    # host check of the stopping rule after every step), on the HA and D of that FP64 analysis;
    # the solve alone is timed
    HA64, D64, _, _ = an64.intermediates()
    r64 = torch.from_numpy(p64.r).to(dev)

    def torch_cg(tol=1e-8, max_iter=1000):
        Z = torch.zeros_like(D64)
        R = D64.clone()
        P = R.clone()
        rr = (R * R).sum(0)
        dn = rr.sqrt()
        it = 0
        while it < max_iter:
            SP = HA64 @ (HA64.T @ P) / (N - 1) + r64[:, None] * P
            alpha = rr / (P * SP).sum(0)
            Z += alpha * P
            R -= alpha * SP
            rr_new = (R * R).sum(0)
            it += 1
            if bool((rr_new.sqrt() <= tol * dn).all()):
                break
            P = R + (rr_new / rr) * P
            rr = rr_new
        return Z, it

    torch_cg()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, torch_iters = torch_cg()
    e1.record(stream)
    torch.cuda.synchronize()
    torch_cg_ms = e0.elapsed_time(e1)

    # accuracy of one timed configuration against the FP64 oracle (exact analysis)
    import oracle
    E = oracle.obs_perturbations(seed, 0, p.r, N)
    an.analyze(Xf, y, seed, 0, out=out)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    err = oracle.rel_frobenius(out.double().cpu().numpy(), ref)
    an64.analyze(X64, y, seed, 0, out=o64)
    err64 = oracle.rel_frobenius(o64.cpu().numpy(), ref)
    an_r.analyze(Xf, y, seed, 0, out=out)
    err_reduced = oracle.rel_frobenius(out.double().cpu().numpy(), ref)
    an_r.close()
    an_s.analyze(Xf, y, seed, 0, out=out)
    err_senkf = oracle.rel_frobenius(out.double().cpu().numpy(), ref)
    err_senkf_oracle = oracle.rel_frobenius(
        out.double().cpu().numpy(),
        oracle.senkf_alg3(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E))
    an_s.close()

    # roofline of the dominant kernel (the persistent CG solve)
    mN = m * N
    it_avg = float(np.mean(iters))
    ref_avg = float(np.mean(refines))
    b_iter = B_ITER(m, N)
    b_ref = B_REF(m, N)
    alg_bytes = it_avg * b_iter + ref_avg * b_ref
    solve_avg_ms = float(np.mean(solve_ms))
    peak, peak_src = _peaks()
    achieved = alg_bytes / (solve_avg_ms / 1e3) / 1e9
    tr = NCU_TRAFFIC.get(args.precision, {})
    traffic = tr.get("bytes") if tr.get("src_sha") == _src_hash(args.precision) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "solve_kernel<float,64,1>" if args.precision == "fp32" else f"solve_mixed_kernel<{args.precision},64>",
                "peak_source": peak_src, "algorithmic_bytes_per_launch": alg_bytes,
                "launch_ms": solve_avg_ms, "cg_iterations": it_avg, "fp64_refreshes": ref_avg}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[args.precision],
            "data": "synthetic (seeded 512x512 GRF ensemble, random point observations)",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "N": N, "tol": 1e-8,
                       "precision": {"fp32": "fp32 CG + double-float residual refresh",
                                     "fp16": "FP16 hi/lo tensor-core contractions (tcgen05) + double-float refresh",
                                     "bf16": "BF16 hi/lo tensor-core contractions (tcgen05) + double-float refresh"}[args.precision],
                       "solver": "CG preconditioned by R" if args.precondition else "plain CG",
                       "l2": "flushed between steps", "status": last_status["status"]},
            "error": {"rel_frobenius_vs_fp64_oracle": err, "fp64_cg_rel_frobenius": err64,
                      "true_relres_max": last_status["true_relres_max"]},
            "torch_fp64_cg_context": {"solve_ms": torch_cg_ms, "iters": torch_iters,
                                      "note": "plain FP64 CG in PyTorch (cuBLAS DGEMM matvecs), solve only; "
                                              "compare with the solve part of fp64_cg"},
            "fp64_cg": {"ms_per_step": fp64_ms, "solve_ms": fp64_solve_ms, "value": 1e3 / fp64_ms, "unit": UNIT,
                        "iters": s64["iters_max"], "speedup_of_value": value / (ws * 1e3 / fp64_ms),
                        "solver": "plain CG, FP64 throughout"},
            "reduced_variant": {"ms_per_step": reduced_ms, "value": 1e3 / reduced_ms, "unit": UNIT,
                                "phases_ms": dict(zip(("gram", "nxn_cg", "update"), reduced_ph)),
                                "cg_iterations": reduced_st["iters_max"], "status": reduced_st["status"],
                                "rel_frobenius_vs_fp64_oracle": err_reduced,
                                "roofline_gram": _gram_roofline(2.0 * m * N * N, reduced_ph[0]),
                                "method": "Algorithm 2 with CG on I + P^T P (N x N), FP32 ensemble, "
                                          "double-float Gram"},
            "senkf_comparator": {"ms_per_step": senkf_ms, "value": 1e3 / senkf_ms, "unit": UNIT,
                                 "phases_ms": dict(zip(("gram", "sum", "update"), senkf_ph)),
                                 "rel_frobenius_vs_exact_enkf": err_senkf,
                                 "rel_frobenius_vs_oracle_senkf": err_senkf_oracle,
                                 "roofline_gram": _gram_roofline(1.0 * m * N * N, senkf_ph[0]),
                                 "method": "Algorithm 3 (diagonal inverse of S, no solve), FP32 ensemble, "
                                           "double-float Gram; an approximation of the EnKF analysis"},
            "fp32_plain_cg": {"ms_per_step": plain32_ms, "value": 1e3 / plain32_ms, "unit": UNIT,
                              "iters": s_plain["iters_max"], "refinements": s_plain["refinements"]},
            "roofline": roofline,
            "e2e": e2e,
            # innovations, (tile images of HA for the tensor-core path,) solve, update
            "gpu_launches": (3 if args.precision == "fp32" else 4) * args.steps,
            "clocks": clk}
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, E)
        line["cpu_baseline_1core"] = cpu_baseline_one_core(seed)
    print(json.dumps(line), flush=True)


def _gen_problem(args):
    import numpy as np
    import synth
    spec, seed, i = args
    return synth.grf_problem(spec["side"], spec["ell"], spec["N"], spec["m"], 0.5, 1.5, seed, dtype=np.float32,
                             sub=1000 + i)


def run_batched(args):
    """256 independent analyses of uneven size (n log-uniform in [4096, 262144], m = n/4,
    N in {16, 32, 64, 128}, GRF ensembles with correlation length U[4, 32], r ~ U[0.5, 1.5])
    in one persistent launch replayed from a CUDA graph; FP32 with Jacobi preconditioning,
    tol 1e-8. value = analyses/s."""
    import multiprocessing as mp
    import numpy as np
    import synth
    ws, rank, local = _dist()
    seed = _rank_seed(args.seed, rank)
    specs = synth.problems.batched_problem_specs(args.batch_count, seed)
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:   # before any GPU call
        probs = pool.map(_gen_problem, [(sp, seed, i) for i, sp in enumerate(specs)])
    gen_s = time.time() - t0
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2606_19224_gb300 as enkf
    ba = enkf.BatchAnalysis([dict(n=p.n, m=p.m, N=p.N, rowptr=p.rowptr, col=p.col, w=p.w, r=p.r) for p in probs],
                            tol=1e-8)
    Xf = [torch.from_numpy(p.Xf).to(dev) for p in probs]
    y = [torch.from_numpy(p.y).to(dev) for p in probs]
    out = [torch.empty_like(x) for x in Xf]
    seeds = [seed + i for i in range(len(probs))]
    if args.reuse_tuned_plan and os.environ.get("ENKF_TUNE_CACHE"):
        tune_ms = None                     # the plan enkf_batch_create read from the cache file
    else:
        tune_ms = ba.tune(Xf, y, seeds, None, out=out)
    plan = ba.plan()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    for k in range(args.warmup):
        ba.analyze(Xf, y, seeds, [k] * len(probs), out=out)
    st = ba.stats()
    if np.any(st["status"] != 0):
        raise SystemExit(f"warm-up batch failed: {st['status']}")
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, refs = [], []
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ba.analyze(Xf, y, seeds, [args.warmup + k] * len(probs), out=out)
        ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    st = ba.stats()
    ms = _max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev, ws)
    count = len(probs)
    value = _job_rate(count * args.steps, ms / 1e3, ws)
    # end to end: pinned host inputs copied in, the batched call, results copied out
    Xh = [torch.from_numpy(p.Xf).pin_memory() for p in probs]
    yh = [torch.from_numpy(p.y).pin_memory() for p in probs]
    Xo = [torch.empty_like(x).pin_memory() for x in Xh]
    e2e_steps = max(2, args.steps // 4)
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        for a, b in zip(Xf, Xh):
            a.copy_(b, non_blocking=True)
        for a, b in zip(y, yh):
            a.copy_(b, non_blocking=True)
        ba.analyze(Xf, y, seeds, [k] * count, out=out)
        for a, b in zip(Xo, out):
            a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dev, ws)
    e2e = {"value": _job_rate(count * e2e_steps, e2e_s, ws), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in Xh) + sum(v.numel() * 8 for v in yh)),
           "d2h_bytes_per_step": int(sum(x.numel() * 4 for x in Xo))}
    if rank != 0:
        return
    # accuracy: a sample of problems against the exact FP64 analysis
    import oracle
    ba.analyze(Xf, y, seeds, [0] * count, out=out)
    torch.cuda.synchronize()
    errs = []
    order = sorted(range(count), key=lambda i: probs[i].m)
    for i in order[::max(1, count // 8)][:8]:
        p = probs[i]
        E = oracle.obs_perturbations(seeds[i], 0, p.r, p.N)
        ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
        errs.append(oracle.rel_frobenius(out[i].double().cpu().numpy(), ref))
    # roofline: algorithmic bytes of all problems of one launch over the launch time
    alg = 0.0
    for i, p in enumerate(probs):
        alg += float(st["iters_max"][i]) * B_ITER(p.m, p.N) + float(st["refinements"][i]) * B_REF(p.m, p.N)
        alg += 4 * p.n * p.N * 2 + 32 * p.m * p.N   # update (X_f in, X_a out); innovations out (HA, B, D, HA and D double-float)
    launch_ms = ms / args.steps
    peak, peak_src = _peaks()
    achieved = alg / (launch_ms / 1e3) / 1e9
    tb = NCU_TRAFFIC_BATCH
    batch_traffic = (tb["bytes"] if (count == tb["problems"] and args.seed == tb["seed"]
                                     and tb["src_sha"] == _src_hash("batch")) else None)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": launch_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded GRF ensembles, random point observations)",
            "config": {"workload": BATCH_WORKLOAD, "problems": count,
                       "n_range": [min(p.n for p in probs), max(p.n for p in probs)],
                       "sum_mN": int(sum(p.m * p.N for p in probs)), "tol": 1e-8,
                       "precision": "fp32 CG + double-float refresh, preconditioned by R",
                       "plan": plan, "tune_ms": tune_ms, "l2": "flushed between steps",
                       "generation_s": gen_s},
            "error": {"rel_frobenius_vs_fp64_oracle_max": max(errs), "sampled_problems": len(errs),
                      "status_ok": int(np.sum(st["status"] == 0))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": batch_traffic, "kernel": "batch_kernel<128>",
                         "peak_source": peak_src, "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms},
            "e2e": e2e, "gpu_launches": args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_mixed(args):
    """The mixed-precision workload: 1024 x 1024 GRF (length 24), N = 128, m = 262,144,
    r ~ U[0.25, 1.0], tol 1e-8. One line per run; `value` is the BF16 tensor-core path
    (split hi/lo operands, FP32 accumulation in TMEM, double-float refresh); FP16, FP32 and
    FP64 (preconditioned and plain) are timed beside it with their errors against the exact
    FP64 oracle analysis."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_2606_19224_gb300 as enkf
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = _rank_seed(args.seed, rank)
    p = synth.workload(MIXED_WORKLOAD, seed, dtype=np.float32)
    n, m, N = p.n, p.m, p.N
    Xf = torch.from_numpy(p.Xf).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    out = torch.empty_like(Xf)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    E = oracle.obs_perturbations(seed, 0, p.r, N) if rank == 0 else None
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E) if rank == 0 else None

    def timed(an, Xd, od, steps, tag):
        for k in range(args.warmup):
            an.analyze(Xd, y, seed, k, out=od)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            an.analyze(Xd, y, seed, k, out=od)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        st = an.stats()
        an.analyze(Xd, y, seed, 0, out=od)
        err = oracle.rel_frobenius(od.double().cpu().numpy(), ref) if rank == 0 else None
        return {"ms_per_step": ms, "value": 1e3 / ms, "iters": st["iters_max"], "refinements": st["refinements"],
                "true_relres_max": st["true_relres_max"], "rel_frobenius_vs_fp64_oracle": err,
                "status": st["status"], "precision": tag}

    clocks = Clocks(local)
    clocks.start()
    res = {}
    for tag, prec in (("bf16", "bf16"), ("fp16", "fp16"), ("fp32", "fp32")):
        an = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision=prec, tol=1e-8, precondition=1)
        res[tag] = timed(an, Xf, out, args.steps, tag)
        an.close()
    clk = clocks.stop()
    X64 = Xf.double()
    o64 = torch.empty_like(X64)
    for tag, pc in (("fp64_pc", 1), ("fp64", 0)):
        an = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision="fp64", tol=1e-8, precondition=pc)
        res[tag] = timed(an, X64, o64, args.fp64_steps, tag)
        an.close()
    ms = _max_over_ranks(res["bf16"]["ms_per_step"], dev, ws)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": _job_rate(1, ms / 1e3, ws), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded 1024x1024 GRF ensemble, random point observations)",
            "config": {"workload": MIXED_WORKLOAD, "n": n, "m": m, "N": N, "tol": 1e-8,
                       "precision": "BF16 hi/lo split operands on tcgen05, FP32 accumulation, double-float refresh",
                       "l2": "flushed between steps"},
            "variants": res, "gpu_launches": 4 * args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="inner-solve precision of the timed path (default workload)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="problems of the batched workload (256 is the benchmark; fewer for profiling)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, BATCH_WORKLOAD, MIXED_WORKLOAD])
    ap.add_argument("--reuse-tuned-plan", action="store_true",
                    help="batched workload: keep the plan enkf_batch_create read from the ENKF_TUNE_CACHE "
                         "file (written by an earlier run's tuner) instead of tuning again")
    ap.add_argument("--precondition", type=int, default=1,
                    help="1: CG preconditioned by R (default, converges in about N steps); 0: plain CG")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == BATCH_WORKLOAD:
        run_batched(args)
    elif args.workload == MIXED_WORKLOAD:
        run_mixed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
