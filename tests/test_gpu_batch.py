"""GPU parity of the batched persistent launch (enkf_batch_*) against the CPU oracle: every
problem of an uneven batch (n, m = n/4, N in {16, 32, 64, 128}, GRF ensembles, R ~ U[0.5, 1.5])
is compared with the exact FP64 analysis (dense Cholesky of S, Eq. matvec_decomp operator)
for the same Philox perturbations; bar 1e-6 relative Frobenius error (the FP32 path's bar)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-6


def _batch(count, seed, n_lo=256, n_hi=16384):
    return synth.batched_problems(count, seed, dtype=np.float32, n_lo=n_lo, n_hi=n_hi)


def _dicts(probs):
    return [dict(n=p.n, m=p.m, N=p.N, rowptr=p.rowptr, col=p.col, w=p.w, r=p.r) for p in probs]


def _device(probs):
    Xf = [torch.from_numpy(np.ascontiguousarray(p.Xf)).cuda() for p in probs]
    y = [torch.from_numpy(p.y).cuda() for p in probs]
    return Xf, y


def _oracle(p, seed, counter):
    E = oracle.obs_perturbations(seed, counter, p.r, p.N)
    return oracle.enkf_exact(p.Xf.astype(np.float64), p.rowptr, p.col, p.w, p.r, p.y, E)


@pytest.fixture(scope="module")
def batch10():
    return _batch(10, seed=11)


@pytest.mark.parametrize("grid_blocks", [0, 12, 1])
def test_batch_matches_oracle(lib, batch10, grid_blocks):
    probs = batch10
    ba = lib.BatchAnalysis(_dicts(probs), grid_blocks=grid_blocks)
    plan = ba.plan()
    assert 1 <= plan["grid"] and (grid_blocks == 0 or plan["grid"] <= grid_blocks)
    Xf, y = _device(probs)
    seeds = [100 + i for i in range(len(probs))]
    counters = [i * 7 for i in range(len(probs))]
    Xa = ba.analyze(Xf, y, seeds, counters)
    st = ba.stats()
    assert np.all(st["status"] == 0), st
    assert np.all(st["relres_max"] <= 1e-8)
    for i, p in enumerate(probs):
        ref = _oracle(p, seeds[i], counters[i])
        err = oracle.rel_frobenius(Xa[i].double().cpu().numpy(), ref)
        assert err <= TOL, (i, p.n, p.m, p.N, err)
    ba.close()


def test_batch_with_teams_and_shared_ctas(lib):
    # one large problem among small ones on a 16-CTA grid: a multi-CTA team plus a queue of
    # several problems served by the free CTA (and by the team's CTAs once they are done)
    probs = _batch(7, seed=5, n_lo=256, n_hi=2048) + synth.batched_problems(1, seed=6, dtype=np.float32,
                                                                           n_lo=60000, n_hi=65536)
    shapes = [(p.n, p.m, p.N) for p in probs]
    plan = lib.batch_plan(shapes, 16, 1.0)
    assert plan["team_size"].max() >= 2 and len(probs) - plan["team_first"][-1] >= 2
    ba = lib.BatchAnalysis(_dicts(probs), grid_blocks=16)
    assert ba.plan()["teams"] == plan["teams"]
    Xf, y = _device(probs)
    seeds = [3] * len(probs)
    Xa = ba.analyze(Xf, y, seeds, None)
    assert np.all(ba.stats()["status"] == 0)
    for i, p in enumerate(probs):
        ref = _oracle(p, 3, 0)
        assert oracle.rel_frobenius(Xa[i].double().cpu().numpy(), ref) <= TOL, i


def test_batch_replay_is_deterministic_and_table_updates(lib, batch10):
    probs = batch10[:6]
    ba = lib.BatchAnalysis(_dicts(probs))
    Xf, y = _device(probs)
    a = [x.clone() for x in ba.analyze(Xf, y, [1] * 6, [2] * 6)]
    b = ba.analyze(Xf, y, [1] * 6, [2] * 6)          # same table: graph replay only
    assert ba.plan()["graphed"] == 1
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    c = ba.analyze(Xf, y, [9] * 6, [2] * 6)          # new seeds: table re-uploaded
    for i, p in enumerate(probs):
        ref = _oracle(p, 9, 2)
        assert oracle.rel_frobenius(c[i].double().cpu().numpy(), ref) <= TOL
    # in place: X_a == X_f
    Xf2 = [x.clone() for x in Xf]
    ba.analyze(Xf2, y, [1] * 6, [2] * 6, out=Xf2)
    for u, v in zip(a, Xf2):
        assert torch.equal(u, v)


def test_batch_matches_single_analysis(lib, batch10):
    probs = batch10[:4]
    ba = lib.BatchAnalysis(_dicts(probs))
    Xf, y = _device(probs)
    Xa = ba.analyze(Xf, y, [5] * 4, [0] * 4)
    for i, p in enumerate(probs):
        an = lib.Analysis(p.n, p.m, p.N, p.rowptr, p.col, p.w, p.r, precision="fp32", precondition=1)
        single = an.analyze(Xf[i], y[i], seed=5, counter=0)
        d = (single.double() - Xa[i].double()).norm() / single.double().norm()
        assert d.item() <= 2 * TOL
        an.close()


def test_batch_tune_and_cache(lib, batch10, tmp_path, monkeypatch):
    probs = batch10[:8]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("ENKF_TUNE_CACHE", str(cache))
    ba = lib.BatchAnalysis(_dicts(probs))
    Xf, y = _device(probs)
    ms = ba.tune(Xf, y, [4] * 8, None)
    assert ms > 0.0
    plan = ba.plan()
    assert plan["alpha"] in (1.0, 0.9, 0.8)
    line = cache.read_text().splitlines()[-1].split()
    assert float(line[1]) == plan["alpha"]
    assert line[2] == "rows" and [int(v) for v in line[3:7]] == plan["row_floors"]
    assert all(f in (64, 128, 256, 512) for f in plan["row_floors"])
    assert len(line) in (7, 7 + len(probs))        # alpha and floors, or with the measured costs
    assert all(float(c) > 0.0 for c in line[7:])
    Xa = ba.analyze(Xf, y, [4] * 8, None)
    for i, p in enumerate(probs):
        assert oracle.rel_frobenius(Xa[i].double().cpu().numpy(), _oracle(p, 4, 0)) <= TOL
    ba.close()
    # a new handle for the same batch rebuilds the cached plan
    ba2 = lib.BatchAnalysis(_dicts(probs))
    plan2 = ba2.plan()
    assert all(plan2[k] == plan[k] for k in ("grid", "teams", "alpha", "row_floors"))
    Xa = ba2.analyze(Xf, y, [4] * 8, None)
    for i, p in enumerate(probs):
        assert oracle.rel_frobenius(Xa[i].double().cpu().numpy(), _oracle(p, 4, 0)) <= TOL
    ba2.close()


def test_batch_times_and_phase_timers(lib, batch10):
    probs = batch10
    ba = lib.BatchAnalysis(_dicts(probs), grid_blocks=12)
    Xf, y = _device(probs)
    with pytest.raises(lib.EnKFError):
        ba.times()                                  # nothing ran yet
    ba.analyze(Xf, y, [6] * 10, None)
    t = ba.times()
    assert np.all(t["start_us"] >= 0.0) and t["start_us"].min() == 0.0
    assert np.all(t["end_us"] > t["start_us"])
    assert np.all(t["team_size"] >= 1) and t["team_size"].max() <= ba.plan()["grid"]
    with pytest.raises(lib.EnKFError, match="phase timers off"):
        ba.times(phases=True)
    ba.set_phase_timing(True)
    Xa = ba.analyze(Xf, y, [6] * 10, None)
    t = ba.times(phases=True)
    dur = t["end_us"] - t["start_us"]
    ph = t["phase_us"]
    assert ph.shape == (10, 8) and np.all(ph >= 0.0)
    assert np.all(ph[:, 1] > 0.0)                     # every solve ran fused passes
    assert np.all(ph.sum(axis=1) <= dur * 1.01 + 1.0)  # the solve lies inside the problem's span
    for i, p in enumerate(probs):                     # timers change nothing in the result
        assert oracle.rel_frobenius(Xa[i].double().cpu().numpy(), _oracle(p, 6, 0)) <= TOL
    ba.set_phase_timing(False)
    ba.analyze(Xf, y, [6] * 10, None)
    with pytest.raises(lib.EnKFError, match="phase timers off"):
        ba.times(phases=True)
    ba.close()


def test_batch_rejects_unsupported(lib, batch10):
    p = _dicts(batch10[:2])
    with pytest.raises(lib.EnKFError):
        lib.BatchAnalysis(p, precondition=0)
    bad = [dict(p[0]), dict(p[1])]
    bad[1]["r"] = -np.abs(bad[1]["r"])
    with pytest.raises(lib.EnKFError, match="problem 1"):
        lib.BatchAnalysis(bad)
