"""Pin the oracle's CLUSTER options (Section 3's closing remark and the contract reading).

* step cap: each execution of PartialGrowth performs at most `step_cap` growing steps; a cap at
  least as long as the longest uncapped growth changes nothing, and a cap of 1 leaves at most one
  step between consecutive stage starts / Delta doublings in the event trace.
* cumulative contract mode: contracted nodes relax with their own bound D_u, so every D_v is the
  length of a real walk from c_v (D_v >= dist_G(c_v, v)), every D stays within the final Delta,
  and the first stage (no contracted node yet) is identical to the default mode's.
"""
import numpy as np
import pytest

import inputs
import oracle

STEP, DOUBLING, FINALIZE, GUARD, START = 0, 1, 2, 3, 4


def graphs():
    out = []
    for side, W, seed in ((12, 100, 1), (20, 1000, 2)):
        e = inputs.grid(side, W, seed)
        out.append(oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=True))
    for scale, seed in ((9, 3), (10, 4)):
        e = inputs.rmat(scale, 8, 1000, seed)
        out.append(oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=True))
    e = inputs.road_mesh(24, 1000, 5)
    out.append(oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=True))
    return out


GRAPHS = graphs()


def growth_lengths(trace):
    # steps of each PartialGrowth execution: runs of step events between starts / doublings / finalizations
    runs, cur = [], 0
    for ev in trace:
        if ev["kind"] == STEP:
            cur += 1
        elif ev["kind"] in (START, DOUBLING, FINALIZE, GUARD):
            if cur:
                runs.append(cur)
            cur = 0
    if cur:
        runs.append(cur)
    return runs


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("mode", [oracle.CONTRACT_RESET, oracle.CONTRACT_CUMULATIVE])
def test_step_cap(gi, mode):
    g = GRAPHS[gi]
    d0 = oracle.delta0(g)
    for tau, seed in ((0.5, 1), (2.0, 7)):
        base = oracle.cluster(g, tau, seed, d0, contract_mode=mode)
        longest = max(growth_lengths(base.trace))
        same = oracle.cluster(g, tau, seed, d0, contract_mode=mode, step_cap=longest)
        assert np.array_equal(same.center, base.center) and np.array_equal(same.D, base.D)
        assert same.stats == base.stats
        one = oracle.cluster(g, tau, seed, d0, contract_mode=mode, step_cap=1)
        assert max(growth_lengths(one.trace)) == 1
        # still a clustering: every node has a center inside its own cluster
        assert all(one.center[int(c)] == c for c in np.unique(one.center))
        if longest > 1:
            capped = oracle.cluster(g, tau, seed, d0, contract_mode=mode, step_cap=longest - 1)
            assert max(growth_lengths(capped.trace)) <= longest - 1


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_cumulative_bounds(gi):
    g = GRAPHS[gi]
    d0 = oracle.delta0(g)
    for tau, seed, cap in ((0.5, 1, 0), (2.0, 7, 0), (1.0, 3, 2)):
        cl = oracle.cluster(g, tau, seed, d0, contract_mode=oracle.CONTRACT_CUMULATIVE, step_cap=cap)
        # every D within the final Delta (the radius bound of the cumulative mode), and each stage's
        # largest D within that stage's Delta (the trace's finalize events: b = the stage's largest D)
        assert int(cl.D.max()) <= cl.stats["delta_end"]
        fin = cl.trace[cl.trace["kind"] == oracle.TRACE_FINALIZE]
        assert (fin["b"].astype(np.int64) <= fin["delta"].astype(np.int64)).all()
        # D_v bounds the true distance from its center; centers sit at 0
        for c in np.unique(cl.center):
            dist = oracle.dijkstra(g, int(c))
            members = np.nonzero(cl.center == c)[0]
            assert np.all(cl.D[members] >= dist[members])
            assert cl.D[int(c)] == 0


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_cumulative_first_stage_is_default(gi):
    # no contracted node exists during the first stage: its events are the default mode's
    g = GRAPHS[gi]
    d0 = oracle.delta0(g)
    a = oracle.cluster(g, 0.5, 11, d0)
    b = oracle.cluster(g, 0.5, 11, d0, contract_mode=oracle.CONTRACT_CUMULATIVE)
    fa = next(i for i, ev in enumerate(a.trace) if ev["kind"] == FINALIZE)
    fb = next(i for i, ev in enumerate(b.trace) if ev["kind"] == FINALIZE)
    assert fa == fb and np.array_equal(a.trace[:fa + 1], b.trace[:fb + 1])
    first = np.array([a.center[v] == b.center[v] and a.D[v] == b.D[v] for v in range(g.n)])
    assert first.sum() >= int(a.trace[fa]["a"])  # at least the nodes frozen by stage 1


def test_cumulative_differs_from_default_somewhere():
    # the option must change the result on some multi-stage workload (a guard against a no-op flag)
    differ = 0
    for g in GRAPHS:
        d0 = oracle.delta0(g)
        a = oracle.cluster(g, 0.5, 1, d0)
        b = oracle.cluster(g, 0.5, 1, d0, contract_mode=oracle.CONTRACT_CUMULATIVE)
        differ += int(not (np.array_equal(a.center, b.center) and np.array_equal(a.D, b.D)))
    assert differ > 0


def test_rejects_unknown_mode():
    g = GRAPHS[0]
    with pytest.raises(RuntimeError):
        oracle.cluster(g, 0.5, 1, oracle.delta0(g), contract_mode=2)
