"""Host-side checks of the batched-launch planner (enkf_batch_plan): no GPU needed."""
import math

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


def check_plan(shapes, G, alpha, plan):
    g, t = plan["grid"], plan["teams"]
    assert 1 <= g <= G and 1 <= t <= g
    ct, cr, ts, tf, order = (plan[k] for k in ("cta_team", "cta_rank", "team_size", "team_first", "order"))
    # every problem exactly once
    assert sorted(order.tolist()) == list(range(len(shapes)))
    # team_first is an offset table into order
    assert tf[0] == 0 and tf[-1] == len(shapes) and np.all(np.diff(tf) >= 1)
    assert ts.sum() == g
    # a team's CTAs are contiguous, ranked 0 .. size-1
    c = 0
    for team in range(t):
        assert np.all(ct[c:c + ts[team]] == team)
        assert cr[c:c + ts[team]].tolist() == list(range(ts[team]))
        c += ts[team]
    # multi-CTA teams hold one problem each, sized by alpha x cost share, >= 64 rows per CTA
    C = sum(cost(*s) for s in shapes)
    for team in range(t):
        probs = order[tf[team]:tf[team + 1]]
        if ts[team] > 1:
            assert len(probs) == 1
            n, m, N = shapes[probs[0]]
            share = G * cost(n, m, N) / C
            assert share >= 1.5
            assert ts[team] == min(math.floor(alpha * share), (m + 63) // 64)
    return ct, cr, ts, tf, order


def test_plan_uneven_batch(ext):
    specs = batched_problem_specs(256, seed=3)
    shapes = [(s["n"], s["m"], s["N"]) for s in specs]
    G = 152
    plan = ext.batch_plan(shapes, G, 1.0)
    ct, cr, ts, tf, order = check_plan(shapes, G, 1.0, plan)
    # LPT bound on the single-CTA teams: max load <= mean load + largest job
    singles = [team for team in range(plan["teams"]) if ts[team] == 1]
    loads = [sum(cost(*shapes[p]) for p in order[tf[k]:tf[k + 1]]) for k in singles]
    jobs = [cost(*shapes[p]) for k in singles for p in order[tf[k]:tf[k + 1]]]
    assert max(loads) <= sum(loads) / len(loads) + max(jobs) + 1e-6 * max(loads)
    assert plan["grid"] >= G - 1  # the whole grid is used


def test_plan_alpha_shrinks_teams(ext):
    shapes = [(262144, 65536, 128)] * 2 + [(4096, 1024, 16)] * 50
    G = 152
    big = ext.batch_plan(shapes, G, 1.0)
    small = ext.batch_plan(shapes, G, 0.55)
    check_plan(shapes, G, 1.0, big)
    check_plan(shapes, G, 0.55, small)
    assert big["team_size"].max() > small["team_size"].max()


def test_plan_degenerate(ext):
    # one problem, one CTA
    p = ext.batch_plan([(100, 25, 16)], 1, 1.0)
    assert p["grid"] == 1 and p["teams"] == 1 and p["order"].tolist() == [0]
    # one large problem takes the grid minus one CTA at most, capped by m / 64 rows
    p = ext.batch_plan([(4096, 1024, 64)], 152, 1.0)
    check_plan([(4096, 1024, 64)], 152, 1.0, p)
    assert p["teams"] == 1 and p["team_size"][0] == 16
    # ten equal problems: shares of 15.2 CTAs each -> ten teams of 15 (m / 64 does not bind)
    shapes = [(65536, 16384, 32)] * 10
    p = ext.batch_plan(shapes, 152, 1.0)
    check_plan(shapes, 152, 1.0, p)
    assert p["teams"] == 10 and p["team_size"].tolist() == [15] * 10
    # the same problems with few rows: teams capped at ceil(m / 64) = 4 CTAs
    shapes = [(1024, 256, 32)] * 10
    p = ext.batch_plan(shapes, 152, 1.0)
    check_plan(shapes, 152, 1.0, p)
    assert p["team_size"].tolist() == [4] * 10


def test_plan_rejects_bad_args(ext):
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 16)], 0, 1.0)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 200)], 8, 1.0)
    with pytest.raises(ext.EnKFError):
        ext.batch_plan([(100, 25, 16)], 8, 0.0)
