"""Served form: continuous batching over an arena.

Each query's result must be the same when it runs alone (one-graph path) and
when it is served in a mix of overlapping queries (integers: bit-exact).
"""
import time

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("phi_gc", "radius", "phi_approx", "k", "stages", "steps", "doublings", "delta_end", "guard_exits",
          "node_updates", "edges_scanned", "quotient_edges", "centers_drawn")


@pytest.fixture(scope="module")
def env():
    import paper_1506_03265_gb300 as cd
    from inputs.workloads import mixture_tau
    cd.load()
    arena = cd.arena_create()
    ids, ns = [], []
    for g in range(18):
        kind, scale, side, sub = inputs.mix_params(5, g)
        e = inputs.rmat(min(scale, 11), 8, 1000, sub) if kind == 0 else inputs.grid(min(side, 80), 1000, sub)
        ids.append(arena.add(e.src, e.dst, e.w, e.n))
        ns.append(arena.graph(ids[-1]).n)
    return cd, arena, ids, [mixture_tau(n) for n in ns], ns


def alone(cd, arena, gid, tau, seed):
    return cd.estimate(cd.quotient_build(cd.cluster(arena.graph(gid), tau, seed)))


def test_mixed_stream_equals_alone(env):
    cd, arena, ids, taus, ns = env
    big = sorted(ns)[-3]  # the three largest graphs go to the one-graph lane
    srv = cd.server_create(arena, ctas=12, big_nodes=big - 1, idle_seconds=2.0)
    rng = np.random.default_rng(1)
    reqs = [(int(g), int(rng.integers(1, 1 << 30))) for g in rng.integers(0, len(ids), 60)]
    tickets = [srv.submit(ids[g], taus[g], seed) for g, seed in reqs]
    got = {}
    t0 = time.time()
    while len(got) < len(tickets) and time.time() - t0 < 60:
        for t in tickets:
            if t not in got:
                r = srv.poll(t)
                if r is not None:
                    got[t] = r
    assert len(got) == len(tickets)
    for (g, seed), t in zip(reqs, tickets):
        ref = alone(cd, arena, ids[g], taus[g], seed)
        assert {f: got[t][f] for f in FIELDS} == {f: ref[f] for f in FIELDS}
    srv.free()


def test_replay_equals_plain_replay(env):
    cd, arena, ids, taus, ns = env
    srv = cd.server_create(arena, ctas=16, idle_seconds=2.0)
    rng = np.random.default_rng(2)
    g = rng.integers(0, len(ids), 150)
    arrivals = np.cumsum(rng.exponential(1 / 3000.0, g.size))
    seeds = rng.integers(1, 1 << 30, g.size)
    res, lat, el = srv.replay([ids[x] for x in g], [taus[x] for x in g], seeds, arrivals)
    assert (lat >= 0).all() and el > 0
    res_p, lat_p, _ = srv.replay([ids[x] for x in g], [taus[x] for x in g], seeds, arrivals, plain=True)
    assert [{f: r[f] for f in FIELDS} for r in res] == [{f: r[f] for f in FIELDS} for r in res_p]
    srv.free()


def test_idle_relaunch_and_capacity(env):
    cd, arena, ids, taus, ns = env
    srv = cd.server_create(arena, ctas=4, capacity=3, idle_seconds=0.05)
    time.sleep(0.3)  # the serving CTAs leave after the idle limit
    ts = [srv.submit(ids[i], taus[i], 7 + i) for i in range(3)]
    for t, i in zip(ts, range(3)):
        t0 = time.time()
        r = None
        while r is None and time.time() - t0 < 30:
            r = srv.poll(t)
        assert r is not None and r["k"] == alone(cd, arena, ids[i], taus[i], 7 + i)["k"]
    with pytest.raises(cd.CldiamError) as ei:
        srv.submit(ids[0], taus[0], 1)
    assert ei.value.status == -6
    srv.free()
