#!/usr/bin/env python3
"""Benchmark of the CGD-EnKF analysis step on GB300.

One step = one full analysis (observation gather + anomalies + perturbed innovations, the
persistent CG solve of S Z = D, and the ensemble update X_a = X_f + A W) through the C ABI
on the synthetic 512x512 Gaussian-random-field workload: n = 262,144 state variables,
N = 64 members, m = 65,536 randomly placed observations, r ~ U[0.5, 1.5], CG tolerance
1e-8 (true relative residual, checked in double-float or FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). `value` is analyses/s summed over ranks (each rank runs its
own independent analyses: weak scaling, no collective on the data path). The timed headline
is CG preconditioned by R with both HA contractions of every step on the tensor cores
(tcgen05, FP16 hi/lo operands, FP32 accumulation), FP32 vectors, FP64 scalars, each step's
sums over the CTAs formed by atomic adds (`--reduce-order 0`: in a fixed order, bitwise
repeatable) and a double-float residual refresh (meets 1e-6 relative Frobenius error against
the FP64 oracle; `--precision fp32` times the FP32 CUDA-core solve instead). On one GPU the
same run then
measures, after the timed region, every other configuration of the method as keys of the
same line:
  c1_variants      the 512x512 workload in plain FP64 CG (the comparison point), FP64 CG
                   preconditioned by R, plain FP32 CG, and the other preconditioned solves
                   (FP32 on the CUDA cores, BF16 / FP16 on the tensor cores)
  reduced_variant, senkf_comparator   the two one-pass variants on the same ensemble
  c2_mixed         1024x1024 GRF, N = 128, m = 262,144: BF16 / FP16 / FP32 / FP64
  c3_batch         256 uneven analyses in one persistent launch (tuned plan, CUDA graph)
  c4_warm_start    the learned CG warm start, trained here, on held-out problems
  c0_l96           200 Lorenz-96 forecast + analysis cycles
  e2b_table5       Example 2b: L96, H = I, N = 100, tridiagonal R, p up to 1e6 (Table 5)
  cpu_baseline(_1core), cpu_plain_fp64_cg   the CPU oracle and the paper's CG on the host
each with its error against the FP64 oracle and the roofline of its solve.
`--impl reference` times the CPU oracle instead (host cores).
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


# ------------------------------------------------------------------ algorithmic work
# The roofline of an analysis (the paper's CG, Sec. 3.3, with the matvec of Eq.
# matvec_decomp): time = max(F / peak_F, B / BW) over the algorithmic flops F and DRAM bytes
# B, with the iteration and refresh counts the run actually took.
#   per CG step:  B = 2 m N s_HA (HA read twice) + 8 m N s_v (x: 1R+1W, r: 2R+1W, p: 2R+1W)
#                 + 2 m 8 (r_i, twice);  F = 4 m N^2 (HA^T p and HA (.))
#   per refresh:  B = 2 m N s_HA + 3 m N s_v (HA twice, Z, D in, residual out)
# s_HA = s_v = 8 (FP64), 4 (FP32); s_HA = 2 for BF16/FP16 HA with FP32 vectors.
S_BYTES = {"fp64": (8, 8), "fp32": (4, 4), "fp16": (2, 4), "bf16": (2, 4)}


def B_ITER(m, N, prec="fp32"):
    s_ha, s_v = S_BYTES[prec]
    return 2 * m * N * s_ha + 8 * m * N * s_v + 16 * m


def B_REF(m, N, prec="fp32"):
    s_ha, s_v = S_BYTES[prec]
    return 2 * m * N * s_ha + 3 * m * N * s_v


def F_ITER(m, N):
    return 4.0 * m * N * N


def B_FUSED(m, N):
    """The same step as one fused FP32 pass of the one-reduction Hestenes-Stiefel form reads and
    writes it (HA read once, x, r and p read and written, r_i read; S p is formed in the pass
    and never stored): 28 m N + 4 m bytes."""
    return 28 * m * N + 4 * m


# Measured on a GB300 with a register-resident FMA loop (152 SMs at 2.07 GHz): FP64 FMA
# 1.20 TFLOP/s, FP32 FMA 74.7 TFLOP/s. Tensor peaks (BF16 = FP16) from MEASURED_PEAKS.json.
FP64_TFLOPS = 1.20
FP32_TFLOPS = 74.7


def _peak_flops(prec):
    if prec == "fp64":
        return FP64_TFLOPS, "FP64 FMA, measured"
    if prec == "fp32":
        return FP32_TFLOPS, "FP32 FMA, measured"
    return _tensor_peak(), "dense BF16/FP16 tensor, measured sustained"


def _tensor_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("bf16_tflops_sustained", 1700.0))
    except OSError:
        return 1700.0


def analysis_roofline(m, N, prec, iters, refreshes, solve_ms, kernel, traffic=None):
    """Roofline of one solve launch on the byte and flop model above."""
    bw, bw_src = _peaks()
    pf, pf_src = _peak_flops(prec)
    B = iters * B_ITER(m, N, prec) + refreshes * B_REF(m, N, prec)
    F = iters * F_ITER(m, N)
    t_b = B / (bw * 1e9)
    t_f = F / (pf * 1e12)
    t = solve_ms / 1e3
    if t_b >= t_f:
        return {"bound": "hbm", "achieved": B / t / 1e9, "peak": bw, "unit": "GB/s", "frac": t_b / t,
                "traffic": traffic, "kernel": kernel, "peak_source": bw_src,
                "algorithmic_bytes_per_launch": B, "algorithmic_flops_per_launch": F,
                "launch_ms": solve_ms, "cg_iterations": iters, "refreshes": refreshes,
                "compute_bound_frac": t_f / t}
    unit = "TFLOP/s"
    return {"bound": "tensor" if prec in ("fp16", "bf16") else "alu", "achieved": F / t / 1e12, "peak": pf,
            "unit": unit, "frac": t_f / t, "traffic": traffic, "kernel": kernel, "peak_source": pf_src,
            "algorithmic_bytes_per_launch": B, "algorithmic_flops_per_launch": F, "launch_ms": solve_ms,
            "cg_iterations": iters, "refreshes": refreshes, "hbm_frac": t_b / t}

# DRAM bytes (read + write) of one solve launch on this workload per precision, from the ncu
# captures summarised under profiles/ (FP32: solve_kernel_fp32_hs_grf512_N64_m65536.md; FP16:
# solve_mixed_kernel_fp16_grf512_N64_m65536.md; both with atomic step sums, the default), with
# the hash of the kernel sources each capture measured; reported as null once those sources
# have changed.
NCU_TRAFFIC = {"fp32": {"bytes": 0.765940e9, "src_sha": "e360a9e69a4aec5f"},
               "fp16": {"bytes": 0.800592e9, "src_sha": "ceff5266981415e8"}}
# DRAM bytes of one batch_kernel launch on the 256-problem batch (seed 1), recorded in
# profiles/batch_kernel_batched256_grf_dram.md for the sources with this hash.
NCU_TRAFFIC_BATCH = {"bytes": 1.436453e12, "problems": 256, "seed": 1, "src_sha": "869cf69968486ece"}
_KERNEL_SOURCES = {
    "fp32": ("kernels_fp.cu", "common.cuh", "cg_device.cuh", "solve_body.cuh"),
    "fp16": ("kernels_tc.cu", "kernels_tc_fp16.cu", "tc_mixed.cuh", "common.cuh", "cg_device.cuh"),
    "bf16": ("kernels_tc.cu", "kernels_tc_bf16.cu", "tc_mixed.cuh", "common.cuh", "cg_device.cuh"),
    "batch": ("kernels_batch.cu", "solve_body.cuh", "innov_device.cuh", "common.cuh", "cg_device.cuh"),
}


def _recorded_traffic(precision, precondition, reduce_order):
    """The captured DRAM bytes of one solve launch on the 512^2 workload, if the capture's
    configuration (CG preconditioned by R, atomic step sums) and kernel sources are these."""
    tr = NCU_TRAFFIC.get(precision)
    if tr is None or precondition != 1 or reduce_order != 1 or tr["src_sha"] != _src_hash(precision):
        return None
    return tr["bytes"]


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


def _gram_roofline(terms, ms, m, N, ens_bytes=4):
    """The Gram pass of the Reduced and sEnKF variants (`terms` products m N^2 or 2 m N^2 per
    launch, reading the observed rows of X_f plus the CSR operator, r and y). The roofline is
    the slower of the products at the FP32 FMA peak and the bytes at HBM bandwidth; the
    issue efficiency of the double-float implementation (12 FP32 operations per product
    against the FP32 lanes x clock) is reported beside it, not as the roofline fraction."""
    bw, bw_src = _peaks()
    t = ms / 1e3
    B = ens_bytes * m * N + 32 * m
    t_f = 2.0 * terms / (FP32_TFLOPS * 1e12)
    t_b = B / (bw * 1e9)
    ops = DF_OPS_PER_TERM * terms
    issue = ops / t / 1e12
    base = {"terms_per_launch": terms, "algorithmic_bytes_per_launch": B, "launch_ms": ms,
            "issue_efficiency": {"achieved": issue, "peak": FP32_OPS_PEAK_T, "unit": "T FP32 op/s",
                                 "frac": issue / FP32_OPS_PEAK_T, "ops_per_term": DF_OPS_PER_TERM}}
    if t_f >= t_b:
        base.update({"bound": "alu", "achieved": 2.0 * terms / t / 1e12, "peak": FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": t_f / t, "peak_source": "FP32 FMA, measured"})
    else:
        base.update({"bound": "hbm", "achieved": B / t / 1e9, "peak": bw, "unit": "GB/s", "frac": t_b / t,
                     "peak_source": bw_src})
    return base


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


def _oracle_loop(p, seed, reps_cap, budget_s):
    """The oracle as it stands, per analysis: the perturbations from its own Philox stream and
    the exact FP64 analysis (Algorithm 2 route, N x N Cholesky), both inside the timed loop,
    as the library draws E inside each analysis."""
    import numpy as np
    import oracle
    X = p.Xf.astype(np.float64)
    t0 = time.perf_counter()
    reps = 0
    while True:
        E = oracle.obs_perturbations(seed, reps, p.r, p.N)
        oracle.enkf_exact(X, p.rowptr, p.col, p.w, p.r, p.y, E)
        reps += 1
        el = time.perf_counter() - t0
        if el > budget_s or reps >= reps_cap:
            return reps, el


def cpu_baseline(problem, seed, budget_s=20.0, reps_cap=8):
    """The CPU oracle on the host cores: a bounded sample of full-size analyses."""
    reps, el = _oracle_loop(problem, seed, reps_cap, budget_s)
    return {"value": reps / el, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{reps} full-size exact analyses ({WORKLOAD}, Algorithm 2 route, FP64 numpy; "
                      f"perturbations drawn by the oracle's Philox stream inside the timed loop) in {el:.1f} s"}


def _child(code, threads=None, timeout=900):
    env = dict(os.environ)
    if threads:
        env.update(OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads), MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=timeout, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_one_core(seed, reps=3):
    """The same oracle on one thread (BLAS and OpenMP limited to 1), in a child process so that
    the limit holds from its first import."""
    code = ("import json, numpy as np, synth, bench\n"
            f"p = synth.workload({WORKLOAD!r}, {int(seed)}, dtype=np.float32)\n"
            f"n, el = bench._oracle_loop(p, {int(seed)}, {int(reps)}, 1e9)\n"
            "print(json.dumps([n, el]))\n")
    n, el = _child(code, threads=1)
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full-size exact analyses ({WORKLOAD}, Algorithm 2 route, same protocol) "
                      f"on one thread in {el:.1f} s"}


def _cpu_cg_timing(p, seed, k1=2, k2=10):
    """Plain FP64 CPU CG (the paper's method, oracle.cgd_enkf: textbook CG on S Z = D with
    the matvec of Eq. matvec_decomp) on the full-size problem, timed at two fixed step
    counts: returns (set-up + update seconds, seconds per CG step)."""
    import numpy as np
    import oracle
    X = p.Xf.astype(np.float64)
    E = oracle.obs_perturbations(seed, 0, p.r, p.N)
    ts = []
    for k in (k1, k2):
        t0 = time.perf_counter()
        oracle.cgd_enkf(X, p.rowptr, p.col, p.w, p.r, p.y, E, fixed_iters=k)
        ts.append(time.perf_counter() - t0)
    per = (ts[1] - ts[0]) / (k2 - k1)
    return max(ts[0] - k1 * per, 0.0), per


def cpu_cg_baseline(p, seed, iters):
    """The paper's method on the CPU: plain FP64 CG (tol 1e-8, stopping rule as the GPU's), on
    all host cores and on one thread; a bounded sample (2 and 10 CG steps) extrapolated to
    the `iters` steps the plain FP64 GPU CG took on the same problem."""
    fixed, per = _cpu_cg_timing(p, seed)
    code = ("import json, numpy as np, synth, bench\n"
            f"p = synth.workload({WORKLOAD!r}, {int(seed)}, dtype=np.float32)\n"
            f"print(json.dumps(bench._cpu_cg_timing(p, {int(seed)})))\n")
    fixed1, per1 = _child(code, threads=1)
    out = {}
    for tag, (f, q, cores) in (("all_cores", (fixed, per, _cores())), ("one_core", (fixed1, per1, 1))):
        t = f + iters * q
        out[tag] = {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle plain FP64 CG",
                    "s_per_cg_step": q, "s_setup_and_update": f, "cg_steps": iters,
                    "sample": f"oracle.cgd_enkf on {WORKLOAD} timed at 2 and 10 CG steps, extrapolated "
                              f"to {iters} steps"}
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands (exact FP64 analysis, perturbations from
    its own Philox stream inside the loop) on the host cores, rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    p = synth.workload(WORKLOAD, args.seed, dtype=np.float32)
    X = p.Xf.astype(np.float64)
    for k in range(args.warmup):
        oracle.enkf_exact(X, p.rowptr, p.col, p.w, p.r, p.y, oracle.obs_perturbations(args.seed, k, p.r, p.N))
    t0 = time.perf_counter()
    for k in range(args.steps):
        E = oracle.obs_perturbations(args.seed, k, p.r, p.N)
        oracle.enkf_exact(X, p.rowptr, p.col, p.w, p.r, p.y, E)
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
                                       f"from the oracle's Philox stream inside the timed loop"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Timer:
    """CUDA-event timing of analyses on the launching stream, L2 flushed before each."""

    def __init__(self, stream, flush):
        self.stream, self.flush = stream, flush

    def analyses(self, an, Xd, y, seed, steps, warmup, out, phases=True, counter0=0):
        import numpy as np
        import torch
        for k in range(warmup):
            an.analyze(Xd, y, seed, counter0 + k, out=out)
        an.set_phase_timing(phases)
        tot, solve, iters, refs = [], [], [], []
        for k in range(steps):
            self.flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            an.analyze(Xd, y, seed, counter0 + warmup + k, out=out)
            e1.record(self.stream)
            torch.cuda.synchronize()
            tot.append(e0.elapsed_time(e1))
            if phases:
                solve.append(an.phase_times()[1])
            st = an.stats()
            iters.append(st["iters_max"])
            refs.append(st["refinements"])
        an.set_phase_timing(False)
        return {"ms_per_step": float(np.mean(tot)), "solve_ms": float(np.mean(solve)) if solve else None,
                "iters": float(np.mean(iters)), "refinements": float(np.mean(refs)), "status": st["status"],
                "true_relres_max": st["true_relres_max"]}


def _err(out, ref):
    import numpy as np
    import oracle
    X = out.double().cpu().numpy()
    return {"rel_frobenius_vs_fp64_oracle": oracle.rel_frobenius(X, ref),
            "max_abs_err_over_max_abs": float(np.max(np.abs(X - ref)) / np.max(np.abs(ref)))}


# how each step's sums over the CTAs are formed (enkf_config.reduce_order)
DTYPE = {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}
PRECISION_NAME = {"fp32": "fp32 CG + double-float residual refresh",
                  "fp16": "FP16 hi/lo tensor-core contractions (tcgen05) + double-float refresh",
                  "bf16": "BF16 hi/lo tensor-core contractions (tcgen05) + double-float refresh"}
REDUCE_NAME = {0: "fixed order (bitwise repeatable)",
               1: "atomic adds (N <= 64; last bits vary from run to run)"}
KERNEL_NAME = {"fp64": "solve_kernel<double>", "fp32": "solve_kernel<float>",
               "fp16": "solve_mixed_kernel<half>", "bf16": "solve_mixed_kernel<bf16>"}


def _variant(enkf, p, prec, pc, timer, Xd, y, seed, steps, warmup, ref, reduce_order=0, traffic=None):
    """One precision / solver variant on problem p: timing, iterations, accuracy and the
    roofline of its solve launch."""
    import torch
    an = enkf.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision=prec, tol=1e-8, precondition=pc,
                       reduce_order=reduce_order)
    out = torch.empty_like(Xd)
    res = timer.analyses(an, Xd, y, seed, steps, warmup, out)
    an.analyze(Xd, y, seed, 0, out=out)
    torch.cuda.synchronize()
    if ref is not None:
        res.update(_err(out, ref))
    res["value"] = 1e3 / res["ms_per_step"]
    res["unit"] = UNIT
    res["solver"] = "CG preconditioned by R" if pc else "plain CG"
    res["reduce_order"] = REDUCE_NAME[reduce_order]
    res["roofline"] = analysis_roofline(p.m, p.N, prec, res["iters"], res["refinements"] if prec != "fp64" else 1,
                                        res["solve_ms"], KERNEL_NAME[prec], traffic)
    an.close()
    return res


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
                       precondition=args.precondition, reduce_order=args.reduce_order)
    an.set_phase_timing(True)
    Xf = torch.from_numpy(p.Xf).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    out = torch.empty_like(Xf)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    timer = Timer(stream, flush)

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

    # ---- the timed region: K analyses of the headline configuration
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

    # ---- end to end through the host-buffer entry point (pinned host memory, copies inside)
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
           "d2h_bytes_per_step": int(Xo.numel() * 4),
           "host_reads_bytes_per_step": int(len(p.col) * N * 4),
           "note": "enkf_analyze_host with pinned buffers: the innovations read the observed rows of X_f "
                   "from host memory (host_reads_bytes_per_step, over the CPU-GPU link, besides the "
                   "copies), X_f is uploaded on a second stream while the solve runs, the update "
                   "writes X_a straight into the pinned output buffer"}

    # ---- roofline of the dominant kernel (the persistent CG solve), live CUDA-event time
    it_avg, ref_avg = float(np.mean(iters)), float(np.mean(refines))
    solve_avg_ms = float(np.mean(solve_ms))
    traffic = _recorded_traffic(args.precision, args.precondition, args.reduce_order)
    roofline = analysis_roofline(m, N, args.precision, it_avg, ref_avg, solve_avg_ms,
                                 KERNEL_NAME[args.precision] + ("<64, preconditioned>" if args.precondition else "<64>"),
                                 traffic)
    roofline["fused_pass_model"] = {
        "bytes_per_launch": it_avg * B_FUSED(m, N) + ref_avg * 56 * m * N,
        "note": "HA read once per step, x, r, p read and written (28 m N + 4 m) and a double-float refresh "
                "of 56 m N bytes: what the fused implementation moves at minimum"}

    prec_name = PRECISION_NAME[args.precision]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic (seeded 512x512 GRF ensemble, random point observations)",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "N": N, "tol": 1e-8, "precision": prec_name,
                       "solver": "CG preconditioned by R" if args.precondition else "plain CG",
                       "reduce_order": REDUCE_NAME[args.reduce_order],
                       "l2": "flushed between steps", "status": last_status["status"]},
            "roofline": roofline, "e2e": e2e,
            # innovations, (tile images of HA for the tensor-core path,) solve, update
            "gpu_launches": (3 if args.precision == "fp32" else 4) * args.steps,
            "clocks": clk}
    if ws > 1 or args.headline_only:
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    # ---- everything below: one GPU, after the timed region
    import oracle
    E = oracle.obs_perturbations(seed, 0, p.r, N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    an.analyze(Xf, y, seed, 0, out=out)
    torch.cuda.synchronize()
    line["error"] = dict(_err(out, ref), true_relres_max=last_status["true_relres_max"])
    an.close()
    t_sec = {}

    # C1 variants: the comparison points (plain FP64 CG, the metric's baseline; FP64 CG
    # preconditioned by R, so that the precision gain is shown apart from the preconditioning
    # gain), plain FP32 CG, and the tensor-core forms
    t0 = time.time()
    X64 = Xf.double()
    c1 = {}
    c1["fp64_plain_cg"] = _variant(enkf, p, "fp64", 0, timer, X64, y, seed, args.fp64_steps, 1, ref)
    c1["fp64_pcg"] = _variant(enkf, p, "fp64", 1, timer, X64, y, seed, args.fp64_steps, 1, ref)
    c1["fp32_plain_cg"] = _variant(enkf, p, "fp32", 0, timer, Xf, y, seed, args.fp64_steps, 1, ref)
    # the headline's precision with the other reduction order, then the other precisions with
    # the headline's order
    other = 1 - args.reduce_order
    c1[args.precision + "_pcg_" + ("atomic" if other else "fixed_order")] = _variant(
        enkf, p, args.precision, 1, timer, Xf, y, seed, max(3, args.steps // 4), 2, ref, reduce_order=other)
    for prec in ("fp32", "fp16", "bf16"):
        if prec != args.precision:
            c1[prec + "_pcg"] = _variant(enkf, p, prec, 1, timer, Xf, y, seed, max(3, args.steps // 4), 2, ref,
                                         reduce_order=args.reduce_order,
                                         traffic=_recorded_traffic(prec, 1, args.reduce_order))
    base = c1["fp64_plain_cg"]["ms_per_step"]
    for k, v in c1.items():
        v["speedup_vs_fp64_plain_cg"] = base / v["ms_per_step"]
    line["speedup_vs_fp64_plain_cg"] = value / (1e3 / base)
    line["speedup_vs_fp64_pcg"] = value / (1e3 / c1["fp64_pcg"]["ms_per_step"])
    line["c1_variants"] = c1

    # the variants built on one Gram pass over the observation rows (FP32 ensemble)
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
    an_r.analyze(Xf, y, seed, 0, out=out)
    err_reduced = _err(out, ref)
    an_r.close()
    an_s = enkf.Analysis(n, m, N, p.rowptr, p.col, p.w, p.r, precision="fp32", variant="senkf")
    senkf_ms, senkf_ph = time_variant(an_s)
    an_s.analyze(Xf, y, seed, 0, out=out)
    err_senkf = oracle.rel_frobenius(out.double().cpu().numpy(), ref)
    err_senkf_oracle = oracle.rel_frobenius(
        out.double().cpu().numpy(), oracle.senkf_alg3(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E))
    an_s.close()
    line["reduced_variant"] = {
        "ms_per_step": reduced_ms, "value": 1e3 / reduced_ms, "unit": UNIT,
        "phases_ms": dict(zip(("gram", "nxn_cg", "update"), reduced_ph)),
        "cg_iterations": reduced_st["iters_max"], "status": reduced_st["status"], **err_reduced,
        "roofline_gram": _gram_roofline(2.0 * m * N * N, reduced_ph[0], m, N),
        "method": "Algorithm 2 with CG on I + P^T P (N x N), FP32 ensemble, double-float Gram"}
    line["senkf_comparator"] = {
        "ms_per_step": senkf_ms, "value": 1e3 / senkf_ms, "unit": UNIT,
        "phases_ms": dict(zip(("gram", "sum", "update"), senkf_ph)),
        "rel_frobenius_vs_exact_enkf": err_senkf, "rel_frobenius_vs_oracle_senkf": err_senkf_oracle,
        "roofline_gram": _gram_roofline(1.0 * m * N * N, senkf_ph[0], m, N),
        "method": "Algorithm 3 (diagonal inverse of S, no solve), FP32 ensemble, double-float Gram; "
                  "an approximation of the EnKF analysis"}
    line["torch_fp64_cg_context"] = _torch_cg_context(enkf, p, X64, y, seed, N, dev, stream)
    t_sec["c1"] = time.time() - t0

    for name, fn in (("c2_mixed", section_c2), ("c3_batch", section_c3), ("c4_warm_start", section_c4),
                     ("c0_l96", section_c0), ("e2b_table5", section_e2b)):
        if name in args.skip:
            continue
        t0 = time.time()
        line[name] = fn(args, enkf, dev, timer)
        t_sec[name] = time.time() - t0
        torch.cuda.empty_cache()

    if not args.no_cpu_baseline:
        t0 = time.time()
        line["cpu_baseline"] = cpu_baseline(p, seed)
        line["cpu_baseline_1core"] = cpu_baseline_one_core(seed)
        line["cpu_plain_fp64_cg"] = cpu_cg_baseline(p, seed, int(round(c1["fp64_plain_cg"]["iters"])))
        t_sec["cpu"] = time.time() - t0
    line["section_wall_s"] = t_sec
    print(json.dumps(line), flush=True)


def _torch_cg_context(enkf, p, X64, y, seed, N, dev, stream):
    """Context only, so that the FP64 comparison point is visibly not a strawman: the same plain
    FP64 CG written with PyTorch (cuBLAS DGEMM for the two contractions of every matvec, a
    host check of the stopping rule after every step), on the HA and D of an FP64 analysis;
    the solve alone is timed."""
    import torch
    an64 = enkf.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp64", tol=1e-8)
    o64 = torch.empty_like(X64)
    an64.analyze(X64, y, seed, 0, out=o64)
    HA64, D64, _, _ = an64.intermediates()
    an64.close()
    r64 = torch.from_numpy(p.r).to(dev)

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
    return {"solve_ms": e0.elapsed_time(e1), "iters": torch_iters,
            "note": "plain FP64 CG in PyTorch (cuBLAS DGEMM matvecs), solve only; compare with the solve part "
                    "of c1_variants.fp64_plain_cg"}


def section_c2(args, enkf, dev, timer):
    """The mixed-precision workload (1024 x 1024 GRF, length 24, N = 128, m = 262,144,
    r ~ U[0.25, 1.0], tol 1e-8): BF16 and FP16 tensor-core contractions (split operands, FP32
    accumulation) with the double-float refresh, FP32, and the FP64 comparison points, each
    against the exact FP64 oracle analysis."""
    import numpy as np
    import torch
    import oracle
    import synth
    seed = args.seed
    p = synth.workload(MIXED_WORKLOAD, seed, dtype=np.float32)
    E = oracle.obs_perturbations(seed, 0, p.r, p.N)
    ref = oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)
    Xf = torch.from_numpy(p.Xf).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    res = {"workload": MIXED_WORKLOAD, "n": p.n, "m": p.m, "N": p.N}
    steps = max(3, min(args.steps, 6))
    X64 = Xf.double()
    if getattr(args, "headline_only", False) and getattr(args, "workload", None) == MIXED_WORKLOAD:
        # the workload alone in one precision (a short run for profiling that one solve)
        prec = args.precision
        res[prec + "_pcg"] = _variant(enkf, p, prec, 1, timer, X64 if prec == "fp64" else Xf, y, seed, steps, 2,
                                      ref)
        return res
    for prec in ("bf16", "fp16", "fp32"):
        res[prec + "_pcg"] = _variant(enkf, p, prec, 1, timer, Xf, y, seed, steps, 2, ref)
    res["fp64_pcg"] = _variant(enkf, p, "fp64", 1, timer, X64, y, seed, 2, 1, ref)
    res["fp64_plain_cg"] = _variant(enkf, p, "fp64", 0, timer, X64, y, seed, 1, 1, ref)
    base = res["fp64_plain_cg"]["ms_per_step"]
    for k in ("bf16_pcg", "fp16_pcg", "fp32_pcg", "fp64_pcg"):
        res[k]["speedup_vs_fp64_plain_cg"] = base / res[k]["ms_per_step"]
        res[k]["speedup_vs_fp64_pcg"] = res["fp64_pcg"]["ms_per_step"] / res[k]["ms_per_step"]
    return res


def _gen_problem(args):
    import numpy as np
    import synth
    spec, seed, i = args
    return synth.grf_problem(spec["side"], spec["ell"], spec["N"], spec["m"], 0.5, 1.5, seed, dtype=np.float32,
                             sub=1000 + i)


def _batch_problems(count, seed):
    import multiprocessing as mp
    import synth
    specs = synth.problems.batched_problem_specs(count, seed)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_problem, [(sp, seed, i) for i, sp in enumerate(specs)])


def _batch_run(args, enkf, dev, timer, probs, seed, steps, warmup, ws=1, barrier=None):
    """Tune, time and check one batched launch; returns (value, ms, the section dict)."""
    import numpy as np
    import torch
    ba = enkf.BatchAnalysis([dict(n=p.n, m=p.m, N=p.N, rowptr=p.rowptr, col=p.col, w=p.w, r=p.r) for p in probs],
                            tol=1e-8)
    Xf = [torch.from_numpy(p.Xf).to(dev) for p in probs]
    y = [torch.from_numpy(p.y).to(dev) for p in probs]
    out = [torch.empty_like(x) for x in Xf]
    seeds = [seed + i for i in range(len(probs))]
    if getattr(args, "reuse_tuned_plan", False) and os.environ.get("ENKF_TUNE_CACHE"):
        tune_ms = None                     # the plan enkf_batch_create read from the cache file
    else:
        tune_ms = ba.tune(Xf, y, seeds, None, out=out)
    plan = ba.plan()
    stream = timer.stream
    barrier = barrier or torch.cuda.synchronize
    for k in range(warmup):
        ba.analyze(Xf, y, seeds, [k] * len(probs), out=out)
    st = ba.stats()
    if np.any(st["status"] != 0):
        raise SystemExit(f"warm-up batch failed: {st['status']}")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    for k in range(steps):
        timer.flush.fill_(float(k))
        ev[k][0].record(stream)
        ba.analyze(Xf, y, seeds, [warmup + k] * len(probs), out=out)
        ev[k][1].record(stream)
    barrier()
    st = ba.stats()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    count = len(probs)
    # end to end: pinned host inputs copied in, the batched call, results copied out
    Xh = [torch.from_numpy(p.Xf).pin_memory() for p in probs]
    yh = [torch.from_numpy(p.y).pin_memory() for p in probs]
    Xo = [torch.empty_like(x).pin_memory() for x in Xh]
    e2e_steps = max(2, steps // 4)
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
    e2e_s = time.perf_counter() - t0
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
        alg += 4 * p.n * p.N * 2 + 3 * 4 * p.m * p.N   # update (X_f in, X_a out); innovations (HA, D written, X_f rows read)
    launch_ms = ms / steps
    peak, peak_src = _peaks()
    achieved = alg / (launch_ms / 1e3) / 1e9
    tb = NCU_TRAFFIC_BATCH
    batch_traffic = (tb["bytes"] if (count == tb["problems"] and seed == tb["seed"]
                                     and tb["src_sha"] == _src_hash("batch")) else None)
    sec = {"workload": BATCH_WORKLOAD, "problems": count, "value": count * steps / (ms / 1e3), "unit": UNIT,
           "ms_per_launch": launch_ms, "steps": steps,
           "n_range": [min(p.n for p in probs), max(p.n for p in probs)],
           "sum_mN": int(sum(p.m * p.N for p in probs)), "plan": plan, "tune_ms": tune_ms,
           "rel_frobenius_vs_fp64_oracle_max": max(errs), "sampled_problems": len(errs),
           "status_ok": int(np.sum(st["status"] == 0)),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": batch_traffic, "kernel": "batch_kernel<128>",
                        "peak_source": peak_src, "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms},
           "e2e": {"value": count * e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in Xh) + sum(v.numel() * 8 for v in yh)),
                   "d2h_bytes_per_step": int(sum(x.numel() * 4 for x in Xo))},
           "gpu_launches": steps}
    ba.close()
    return sec, ms


def section_c3(args, enkf, dev, timer):
    """256 analyses of uneven size in one persistent launch replayed from a CUDA graph, plan
    tuned on the batch."""
    t0 = time.time()
    probs = _batch_problems(args.batch_count, args.seed)
    gen_s = time.time() - t0
    sec, _ = _batch_run(args, enkf, dev, timer, probs, args.seed, steps=3, warmup=2)
    sec["generation_s"] = gen_s
    return sec


def section_c4(args, enkf, dev, timer):
    """Learned warm start on the 512 x 512 workload shapes: train the MLP (1,024-row sketch + N
    projections -> 3 x 512 GELU -> N) with the library's kernels on pairs from the method's own
    solves, then time held-out analyses from the zero start and from the learned start."""
    from paper_2606_19224_gb300 import warm_train
    cfg = dict(warm_train.FULL)
    cfg.update(train_seeds=args.warm_train_seeds, draws=8, test_seeds=4, epochs=40)
    res, _ = warm_train.run(cfg, log=lambda s: None)
    ev = res["eval"]
    return {"train_problems": cfg["train_seeds"] * cfg["draws"], "pairs": res["pairs"],
            "loss_first": res["loss_first"], "loss_last": res["loss_last"],
            "collect_s": res["collect_s"], "train_s": res["train_s"],
            "iters_mean_zero": res["iters_mean_zero"], "iters_mean_learned": res["iters_mean_learned"],
            "ms_zero": res["ms_zero"], "ms_learned": res["ms_learned"],
            "speedup": res["ms_zero"] / res["ms_learned"],
            "rel_diff_zero_vs_learned_max": max(r["rel_diff_zero_vs_learned"] for r in ev),
            "warm_fallbacks": sum(r["learned"]["warm_fallbacks"] for r in ev),
            "status": [r["learned"]["status"] for r in ev], "held_out_seeds": len(ev),
            "judge": "a start is kept only if its true residual is at most ||d_j|| (warm_accept = 0)",
            "accept_all_finite": {
                "iters_mean": res["iters_mean_learned_accept"], "ms": res["ms_learned_accept"],
                "speedup": res["ms_zero"] / res["ms_learned_accept"],
                "rel_diff_zero_vs_learned_max": max(r["rel_diff_zero_vs_learned_accept"] for r in ev),
                "true_relres_max": max(r["learned_accept"]["true_relres_max"] for r in ev),
                "start_relres_max": max(r["learned_accept"]["warm_relres_max"] for r in ev),
                "refinements": [r["learned_accept"]["refinements"] for r in ev],
                "refinements_zero_start": [r["zero"]["refinements"] for r in ev],
                "status": [r["learned_accept"]["status"] for r in ev],
                "note": "every finite start kept (warm_accept = 1); the result is certified by the same "
                        "double-float true residual <= tol"}}


def section_c0(args, enkf, dev, timer):
    """Lorenz-96 cycling (n = 40, N = 20, m = 20, R = I, FP64, tol 1e-10): 200 forecast +
    analysis cycles with the analysis on the GPU and the forecast on the host; the oracle
    analyses the same forecast each cycle (lockstep error), and the same 200 cycles with the
    oracle's analysis give the CPU rate."""
    import numpy as np
    import torch
    import oracle
    import synth
    cycles = 200

    def run(gpu):
        cyc = synth.L96Cycle(seed=args.seed)
        an = enkf.Analysis(40, cyc.col.size, 20, cyc.rowptr, cyc.col, cyc.w, cyc.r, precision="fp64",
                           tol=1e-10) if gpu else None
        yd = torch.empty(cyc.col.size, dtype=torch.float64, device=dev) if gpu else None
        Xd = torch.empty((40, 20), dtype=torch.float64, device=dev) if gpu else None
        err, an_s = 0.0, 0.0
        t0 = time.perf_counter()
        for k in range(cycles):
            cyc.forecast()
            y = cyc.observe()
            ta = time.perf_counter()
            if gpu:
                Xd.copy_(torch.from_numpy(cyc.ensemble))
                yd.copy_(torch.from_numpy(y))
                Xa = an.analyze(Xd, yd, seed=99, counter=k).cpu().numpy()
            else:
                Xa = oracle.enkf_alg1(cyc.ensemble, cyc.rowptr, cyc.col, cyc.w, cyc.r, y,
                                      oracle.obs_perturbations(99, k, cyc.r, 20))
            an_s += time.perf_counter() - ta
            if gpu and k % 20 == 0:
                ref = oracle.enkf_alg1(cyc.ensemble, cyc.rowptr, cyc.col, cyc.w, cyc.r, y,
                                       oracle.obs_perturbations(99, k, cyc.r, 20))
                err = max(err, oracle.rel_frobenius(Xa, ref))
            cyc.ensemble = np.ascontiguousarray(Xa)
        el = time.perf_counter() - t0
        rmse = float(np.sqrt(np.mean((cyc.ensemble.mean(axis=1) - cyc.truth) ** 2)))
        status = an.stats()["status"] if gpu else "ok"
        return el, an_s, err, rmse, status

    el, an_s, err, rmse, status = run(True)
    el_c, an_c, _, rmse_c, _ = run(False)
    return {"cycles": cycles, "cycles_per_s": cycles / el, "analyses_per_s": cycles / an_s,
            "analysis_ms": 1e3 * an_s / cycles, "rel_frobenius_vs_oracle_max_sampled": err,
            "final_rmse_vs_truth": rmse, "status": status,
            "oracle": {"cycles_per_s": cycles / el_c, "analyses_per_s": cycles / an_c, "cores": _cores(),
                       "final_rmse_vs_truth": rmse_c},
            "note": "analysis on the GPU (host copies included), forecast (RK4) on the host; the analyses "
                    "are launch-bound at this size"}


def section_e2b(args, enkf, dev, timer):
    """Example 2b (Table 5): Lorenz-96 with H = I, N = 100, tridiagonal Toeplitz R (sigma = 0.3,
    rho = 0.2), one analysis per p in FP64: EnKF-Reduced (the Reduced analysis run to
    convergence), CGD-EnKF-Reduced with r = 1..5 CG steps and the sEnKF comparator, each timed
    on the GPU and its error against EnKF-Reduced reported beside the paper's printed value."""
    import numpy as np
    import torch
    import oracle
    import synth
    printed = {}
    with open(os.path.join(ROOT, "tests", "golden", "table5_cgd_enkf_reduced.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                pp, r, v = line.split()
                printed[(int(pp), int(r))] = float(v)
    out = {}
    for p in args.e2b_sizes:
        t0 = time.time()
        P = synth.l96_tridiag_problem(p, 100, seed=args.seed)
        gen_s = time.time() - t0
        Xf = torch.from_numpy(P.Xf).to(dev)
        y = torch.from_numpy(P.y).to(dev)
        Xa = torch.empty_like(Xf)

        def timed(an, reps=5):
            an.analyze(Xf, y, out=Xa)
            torch.cuda.synchronize()
            ms = []
            for k in range(reps):
                timer.flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(timer.stream)
                an.analyze(Xf, y, out=Xa)
                e1.record(timer.stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return float(np.median(ms)), Xa.cpu().numpy()

        def mk(**cfg):
            return enkf.Analysis(p, p, 100, P.rowptr, P.col, P.w, P.r, r_off=P.r_off, precision="fp64",
                                 perturb_obs=0, **cfg)

        ms_ref, exact = timed(mk(variant="reduced", tol=1e-13))
        row = {"enkf_reduced_ms": ms_ref, "generation_s": gen_s}
        if p <= 100000:
            row["enkf_reduced_vs_oracle"] = oracle.rel_frobenius(
                exact, oracle.enkf_alg2(P.Xf, P.rowptr, P.col, P.w, P.r, P.y, None, r_off=P.r_off))
        for r in range(1, 6):
            ms, X = timed(mk(variant="reduced", fixed_iters=r))
            row[f"cgd_reduced_r{r}"] = {"ms": ms, "rel_err_vs_enkf_reduced": oracle.rel_frobenius(X, exact),
                                         "paper": printed.get((p, r))}
        ms, X = timed(mk(variant="senkf"))
        row["senkf"] = {"ms": ms, "rel_err_vs_enkf_reduced": oracle.rel_frobenius(X, exact),
                        "paper": printed.get((p, 0))}
        out[str(p)] = row
        del Xf, Xa
        torch.cuda.empty_cache()
    out["note"] = ("FP64 on one GB300; the paper's times are on 50 CPU cores (MPI); errors against the converged "
                   "Reduced analysis (EnKF-Reduced) next to the printed Table 5 values")
    return out


def run_batched(args):
    """The batched workload alone: 256 independent analyses of uneven size (n log-uniform in
    [4096, 262144], m = n/4, N in {16, 32, 64, 128}, GRF ensembles with correlation length
    U[4, 32], r ~ U[0.5, 1.5]) in one persistent launch replayed from a CUDA graph; FP32 with
    Jacobi preconditioning, tol 1e-8. value = analyses/s summed over ranks."""
    import torch
    ws, rank, local = _dist()
    seed = _rank_seed(args.seed, rank)
    t0 = time.time()
    probs = _batch_problems(args.batch_count, seed)        # spawn pool, before any GPU call
    gen_s = time.time() - t0
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2606_19224_gb300 as enkf
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    timer = Timer(torch.cuda.current_stream(), flush)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    sec, ms = _batch_run(args, enkf, dev, timer, probs, seed, args.steps, args.warmup, ws, barrier)
    clk = clocks.stop()
    ms = _max_over_ranks(ms, dev, ws)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": _job_rate(len(probs) * args.steps, ms / 1e3, ws), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded GRF ensembles, random point observations)",
            "config": {"workload": BATCH_WORKLOAD, "problems": len(probs), "l2": "flushed between steps",
                       "generation_s": gen_s},
            "roofline": sec.pop("roofline"), "e2e": sec.pop("e2e"), "gpu_launches": args.steps,
            "clocks": clk, "batch": sec}
    print(json.dumps(line), flush=True)


def run_mixed(args):
    """The mixed-precision workload alone (see section_c2): `value` is the BF16 tensor-core
    path; with --headline-only, only the --precision solve is run and reported (a short run,
    e.g. for profiling that one solve)."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2606_19224_gb300 as enkf
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    timer = Timer(torch.cuda.current_stream(), flush)
    clocks = Clocks(local)
    clocks.start()
    res = section_c2(args, enkf, dev, timer)
    clk = clocks.stop()
    key = args.precision + "_pcg" if args.headline_only else "bf16_pcg"
    ms = _max_over_ranks(res[key]["ms_per_step"], dev, ws)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": _job_rate(1, ms / 1e3, ws), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[key[:4]],
            "data": "synthetic (seeded 1024x1024 GRF ensemble, random point observations)",
            "config": {"workload": MIXED_WORKLOAD, "n": res["n"], "m": res["m"], "N": res["N"], "tol": 1e-8,
                       "precision": PRECISION_NAME[key[:4]], "l2": "flushed between steps"},
            "roofline": res[key]["roofline"], "variants": res, "gpu_launches": 4 * args.steps,
            "clocks": clk}
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
    ap.add_argument("--headline-only", action="store_true",
                    help="only the timed headline configuration and its end-to-end number")
    ap.add_argument("--skip", default="", help="comma-separated sections to leave out of the default run: "
                                               "c2_mixed, c3_batch, c4_warm_start, c0_l96, e2b_table5")
    ap.add_argument("--e2b-sizes", type=lambda v: [int(x) for x in v.split(",")], default=[1000, 10000, 100000, 1000000],
                    help="state sizes p of the Example 2b (Table 5) section")
    ap.add_argument("--warm-train-seeds", type=int, default=40,
                    help="ensembles (x 8 observation draws) the learned warm start trains on in the default run")
    ap.add_argument("--reduce-order", type=int, default=1, choices=[0, 1],
                    help="1 sums each CG step over the CTAs by atomic adds (one grid barrier per step; "
                         "N <= 64), 0 in a fixed order (bitwise repeatable)")
    ap.add_argument("--precision", default="fp16", choices=["fp32", "fp16", "bf16"],
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
    args.skip = set(x for x in args.skip.split(",") if x)
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
