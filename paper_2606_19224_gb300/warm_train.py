"""Training and evaluation of the learned CG warm start, driven through the library's C ABI
(every arithmetic step runs in its kernels: analyses, feature extraction, MLP forward,
backward and Adam). Pairs (features of d_j, target c_j = W e_j / s_j) come from the
method's own solves on seeded synthetic ensembles; evaluation compares CG iterations and
analysis time with and without the learned start on held-out seeds.

    python -m paper_2606_19224_gb300.warm_train --out warm_results.json

runs the full-size case (512 x 512 GRF, N = 64, m = 65,536, sketch 1,024, 3 x 512 GELU
layers, 20,480 training pairs from 320 analyses over 40 ensembles); --small runs a
seconds-long case.
"""
import argparse
import json
import time

import numpy as np

from . import Analysis, MlpShape, mlp_param_count, mlp_standardize, mlp_train_epoch, mlp_trained_count


def _problem(side, ell, N, m, seed, draw):
    import synth
    # ensemble, observations and perturbation stream from (seed, draw)
    return synth.grf_problem(side, ell, N, m, 0.5, 1.5, seed, dtype=np.float32, sub=draw)


def _problem_args(a):
    return _problem(*a)


def collect_pairs(cfg, seeds, draws, K, log=None, workers=8):
    """Run one FP32 analysis per (seed, draw) (inputs generated by a spawn pool while the GPU
    works); return device F [P][K+N], T [P][N]."""
    import multiprocessing as mp
    import torch
    Fs, Ts = [], []
    jobs = [(cfg["side"], cfg["ell"], cfg["N"], cfg["m"], s, d) for s in seeds for d in range(draws)]
    an = None
    with mp.get_context("spawn").Pool(workers) as pool:
        for q, p in enumerate(pool.imap(_problem_args, jobs)):
            s, d = jobs[q][4], jobs[q][5]
            if an is None:
                an = Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1,
                              tol=cfg["tol"])
            else:
                an.close()
                an = Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1,
                              tol=cfg["tol"])
            an.analyze(torch.from_numpy(p.Xf).cuda(), torch.from_numpy(p.y).cuda(), seed=1000 * s + d, counter=d)
            F, T = an.warm_features(K)
            Fs.append(F)
            Ts.append(T)
            if log and (q + 1) % max(1, len(jobs) // 10) == 0:
                log(f"pairs: {len(Fs) * cfg['N']}")
    if an is not None:
        an.close()
    return torch.cat(Fs), torch.cat(Ts)


def train(shape, F, T, epochs, batch, lr, seed, log=None):
    """Minibatch Adam on (F, T); returns (params, per-epoch mean losses)."""
    import torch
    import synth.mlp_init as mi
    dims = (shape.in_dim, shape.hidden, shape.layers, shape.out_dim)
    params = torch.from_numpy(mi.init_params(*dims, seed=seed)).cuda()
    mlp_standardize(shape, params, F, T)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    rng = np.random.default_rng(seed)
    P = F.shape[0]
    hist, step = [], 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(P).astype(np.int32)).cuda()
        # cosine learning-rate decay over the epochs
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(1, epochs)))
        losses = mlp_train_epoch(shape, params, m, v, F, T, perm, batch, step, float(lr_ep))
        step += P // batch
        hist.append(float(losses.mean().item()))
        if log and (ep % max(1, epochs // 10) == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return params, hist


def evaluate(cfg, shape, params, seeds, K, reps=5):
    """Per held-out problem: mean / max CG iterations over columns and analysis time (ms),
    zero start vs learned start, plus the learned start's true residual. The learned start is
    judged both ways: "learned" keeps a column's start only if its true residual is at most
    ||d_j|| (warm_accept = 0), "learned_accept" keeps every finite start (warm_accept = 1)."""
    import torch
    out = []
    for s in seeds:
        p = _problem(cfg["side"], cfg["ell"], cfg["N"], cfg["m"], s, 0)
        Xf = torch.from_numpy(p.Xf).cuda()
        y = torch.from_numpy(p.y).cuda()
        row = dict(seed=s)
        for mode in ("zero", "learned", "learned_accept"):
            an = Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1,
                          tol=cfg["tol"], warm_start=0 if mode == "zero" else 1,
                          warm_accept=1 if mode == "learned_accept" else 0)
            if mode != "zero":
                an.set_warm_model(shape, params)
            Xa = an.analyze(Xf, y, seed=77 + s, counter=0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                an.analyze(Xf, y, seed=77 + s, counter=0, out=Xa)
            e1.record()
            torch.cuda.synchronize()
            an.set_phase_timing(True)
            an.analyze(Xf, y, seed=77 + s, counter=0, out=Xa)
            ph = an.phase_times()
            an.set_phase_timing(False)
            st = an.stats()
            it, _, _ = an.column_stats()
            row[mode] = dict(iters_mean=float(np.mean(it)), iters_max=int(np.max(it)),
                             ms=e0.elapsed_time(e1) / reps, phase_ms=[float(v) for v in ph],
                             refinements=st["refinements"], true_relres_max=st["true_relres_max"],
                             warm_relres_max=st["warm_relres_max"], warm_fallbacks=st["warm_fallbacks"],
                             status=st["status"])
            row[mode + "_Xa"] = Xa
            an.close()
        for mode in ("learned", "learned_accept"):
            d = (row["zero_Xa"].double() - row[mode + "_Xa"].double()).norm() / row["zero_Xa"].double().norm()
            row["rel_diff_zero_vs_" + mode] = float(d.item())
        del row["zero_Xa"], row["learned_Xa"], row["learned_accept_Xa"]
        out.append(row)
    return out


FULL = dict(side=512, ell=16.0, N=64, m=65536, tol=1e-8, K=1024, hidden=512, layers=3, train_seeds=40, draws=8,
            test_seeds=6, epochs=60, batch=256, lr=1e-3)
SMALL = dict(side=64, ell=6.0, N=32, m=1024, tol=1e-8, K=128, hidden=128, layers=3, train_seeds=24, draws=4,
             test_seeds=4, epochs=40, batch=64, lr=2e-3)


def run(cfg, log=print):
    K, N = cfg["K"], cfg["N"]
    shape = MlpShape(K + N, cfg["hidden"], cfg["layers"], N)
    t0 = time.time()
    F, T = collect_pairs(cfg, list(range(100, 100 + cfg["train_seeds"])), cfg["draws"], K, log)
    t1 = time.time()
    params, hist = train(shape, F, T, cfg["epochs"], cfg["batch"], cfg["lr"], seed=1, log=log)
    t2 = time.time()
    ev = evaluate(cfg, shape, params, list(range(900, 900 + cfg["test_seeds"])), K)
    res = dict(config=cfg, pairs=int(F.shape[0]), params=mlp_param_count(shape),
               trained_params=mlp_trained_count(shape), loss_first=hist[0], loss_last=hist[-1],
               loss_history=hist, collect_s=t1 - t0, train_s=t2 - t1, eval=ev)
    for mode in ("zero", "learned", "learned_accept"):
        res["iters_mean_" + mode] = float(np.mean([r[mode]["iters_mean"] for r in ev]))
        res["ms_" + mode] = float(np.mean([r[mode]["ms"] for r in ev]))
    return res, params


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--epochs", type=int, default=None)
    a = ap.parse_args()
    cfg = dict(SMALL if a.small else FULL)
    if a.epochs:
        cfg["epochs"] = a.epochs
    res, params = run(cfg)
    s = json.dumps({k: v for k, v in res.items() if k != "loss_history"}, indent=1)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
        np.save(a.out.rsplit(".", 1)[0] + "_params.npy", params.cpu().numpy())


if __name__ == "__main__":
    main()
