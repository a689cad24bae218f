"""Host-side checks of the batched-launch planner (enkf_batch_plan): no GPU needed.

Contract (include/enkf.h): cost c = m N^2 (N + 8) + 2 n N^2, a team of k CTAs takes
c / k^alpha, problems costlier than the makespan target get a team of 2 <= k <= ceil(m / 64)
CTAs, the rest form a shared queue (longest first) served by whichever CTA is free first: the
CTAs outside teams from the start, each team's CTAs once its problem is done. The target is
the smallest feasible one. The makespan below is an independent event simulation of that
queue."""
import heapq

import numpy as np
import pytest

from synth.problems import batched_problem_specs


@pytest.fixture(scope="module")
def ext():
    import paper_2606_19224_gb300 as ext
    ext.load()
    return ext


def cost(n, m, N):
    return m * N * N * (N + 8.0) + 2.0 * n * N * N


def simulate(shapes, plan, alpha):
    """Finish time of every CTA: team problems first, then the queue taken in order by the
    CTA that is free first."""
    ts, tf, order = plan["team_size"], plan["team_first"], plan["order"]
    free = []
    for t in range(plan["teams"]):
        done = sum(cost(*shapes[p]) for p in order[tf[t]:tf[t + 1]]) / ts[t] ** alpha
        free += [done] * int(ts[t])
    heapq.heapify(free)
    for p in order[tf[-1]:]:
        heapq.heappush(free, heapq.heappop(free) + cost(*shapes[p]))
    return np.array(sorted(free))


def lower_bound(shapes, G, alpha):
    caps = [max(1, min(G, (m + 63) // 64)) for _, m, _ in shapes]
    total = sum(cost(*s) for s in shapes)
    return max(total / G, max(cost(*s) / c ** alpha for s, c in zip(shapes, caps)))


def check_plan(shapes, G, alpha, plan):
    g, t = plan["grid"], plan["teams"]
    assert 1 <= g <= G and 1 <= t <= g
    ct, cr, ts, tf, order = (plan[k] for k in ("cta_team", "cta_rank", "team_size", "team_first", "order"))
    assert sorted(order.tolist()) == list(range(len(shapes)))          # every problem once
    assert tf[0] == 0 and tf[-1] <= len(shapes) and np.all(np.diff(tf) >= 0)
    assert ts.sum() == g
    c = 0
    for team in range(t):                                               # contiguous, ranked
        assert np.all(ct[c:c + ts[team]] == team)
        assert cr[c:c + ts[team]].tolist() == list(range(ts[team]))
        c += ts[team]
    for team in range(t):
        probs = order[tf[team]:tf[team + 1]]
        if ts[team] > 1:                                                # one problem, capped team
            assert len(probs) == 1
            assert ts[team] <= (shapes[probs[0]][1] + 63) // 64
        else:                                                           # a free CTA
            assert len(probs) == 0
    qc = [cost(*shapes[p]) for p in order[tf[-1]:]]
    assert all(a >= b for a, b in zip(qc, qc[1:]))                      # queue: longest first
    return simulate(shapes, plan, alpha)


# with alpha < 1 the bound total/G (perfect scaling) is loose, hence the wider factor
@pytest.mark.parametrize("count,alpha,factor", [(256, 1.0, 1.2), (256, 0.9, 1.5), (24, 1.0, 1.2),
                                                (24, 0.8, 2.0), (7, 1.0, 1.2)])
def test_plan_uneven_batch_near_lower_bound(ext, count, alpha, factor):
    specs = batched_problem_specs(count, seed=1)
    shapes = [(s["n"], s["m"], s["N"]) for s in specs]
    G = 152
    plan = ext.batch_plan(shapes, G, alpha)
    times = check_plan(shapes, G, alpha, plan)
    lb = lower_bound(shapes, G, alpha)
    assert times.max() <= factor * lb, (times.max() / lb)
    assert plan["team_first"][-1] < count                               # the queue is used


def test_plan_degenerate(ext):
    # one problem, one CTA: a free CTA and the problem in the queue
    p = ext.batch_plan([(100, 25, 16)], 1, 1.0)
    assert p["grid"] == 1 and p["teams"] == 1 and p["order"].tolist() == [0]
    assert p["team_first"].tolist() == [0, 0]
    # one large problem: as many CTAs as its rows allow (64 rows per CTA)
    p = ext.batch_plan([(4096, 1024, 64)], 152, 1.0)
    check_plan([(4096, 1024, 64)], 152, 1.0, p)
    assert p["teams"] == 1 and p["team_size"][0] == 16
    # ten equal problems share the grid evenly (15 or 16 CTAs each, all 152 used)
    shapes = [(65536, 16384, 32)] * 10
    p = ext.batch_plan(shapes, 152, 1.0)
    check_plan(shapes, 152, 1.0, p)
    assert p["teams"] == 10 and p["grid"] == 152 and set(p["team_size"].tolist()) <= {15, 16}
    # the same problems with few rows: teams capped at ceil(m / 64) = 4 CTAs
    shapes = [(1024, 256, 32)] * 10
    p = ext.batch_plan(shapes, 152, 1.0)
    check_plan(shapes, 152, 1.0, p)
    assert p["team_size"].tolist() == [4] * 10
    # many tiny problems: all in the queue on 152 free CTAs, which finish within one
    # problem's time of each other
    shapes = [(256, 64, 16)] * 500
    p = ext.batch_plan(shapes, 152, 1.0)
    done = check_plan(shapes, 152, 1.0, p)
    assert p["team_size"].max() == 1 and p["teams"] == 152 and p["team_first"][-1] == 0
    assert done.max() - done.min() <= cost(*shapes[0]) * (1 + 1e-12)
    # fewer problems than CTAs: one free CTA per problem, no idle CTAs in the grid
    shapes = [(256, 64, 16)] * 5
    p = ext.batch_plan(shapes, 152, 1.0)
    check_plan(shapes, 152, 1.0, p)
    assert p["grid"] == 5


def test_plan_rejects_bad_args(ext):
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 16)], 0, 1.0)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 200)], 8, 1.0)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 16)], 8, 0.0)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 16)], 8, 1.5)


def test_row_floors_cap_the_teams(ext):
    """A row floor f for an N class caps that class's teams at ceil(m / f) CTAs; the other
    classes keep the default of 64 rows; every plan still covers each problem once."""
    specs = batched_problem_specs(64, seed=3)
    shapes = [(s["n"], s["m"], s["N"]) for s in specs]
    cls = lambda N: 0 if N <= 16 else (1 if N <= 32 else (2 if N <= 64 else 3))
    for floors in ([64, 64, 64, 512], [256, 128, 512, 64], [1000, 1000, 1000, 1000]):
        plan = ext.batch_plan(shapes, 152, 1.0, row_floors=floors)
        check_plan(shapes, 152, 1.0, dict(plan))
        ts, tf, order = plan["team_size"], plan["team_first"], plan["order"]
        for t in range(plan["teams"]):
            for p in order[tf[t]:tf[t + 1]]:
                n, m, N = shapes[p]
                assert ts[t] <= max(1, -(-m // floors[cls(N)]))
    # a floor that forbids every team sends every problem to the queue
    big = ext.batch_plan(shapes, 152, 1.0, row_floors=[10 ** 9] * 4)
    assert all(big["team_size"] == 1)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan(shapes, 152, 1.0, row_floors=[64, 0, 64, 64])
