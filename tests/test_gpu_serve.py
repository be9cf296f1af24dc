"""Served form: continuous batching over an arena.

Each query's result must be the same when it runs alone (one-graph path) and
when it is served in a mix of overlapping queries (integers: bit-exact).
"""
import time

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("phi_gc", "radius", "phi_approx", "k", "stages", "steps", "doublings", "delta_end", "guard_exits",
          "node_updates", "edges_scanned", "quotient_edges", "centers_drawn")
# every field the oracle defines the same way (edges_scanned counts the GPU's frontier entries, while the
# oracle re-reads every relaxer's adjacency at every step)
ORACLE_FIELDS = tuple(f for f in FIELDS if f != "edges_scanned")
EDGES = []  # edge lists of the arena's graphs, in arena order


@pytest.fixture(scope="module")
def env():
    import paper_1506_03265_gb300 as cd
    from inputs.workloads import mixture_tau
    cd.load()
    arena = cd.arena_create()
    ids, ns, edges = [], [], []
    for g in range(18):
        kind, scale, side, sub = inputs.mix_params(5, g)
        e = inputs.rmat(min(scale, 11), 8, 1000, sub) if kind == 0 else inputs.grid(min(side, 80), 1000, sub)
        ids.append(arena.add(e.src, e.dst, e.w, e.n))
        ns.append(arena.graph(ids[-1]).n)
        edges.append(e)
    EDGES[:] = edges
    return cd, arena, ids, [mixture_tau(n) for n in ns], ns


def oracle_result(e, tau, seed):
    """The whole method on the CPU oracle, as a dict over ORACLE_FIELDS."""
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    ores, ocl, oq = oracle.cldiam(og, tau, seed)
    out = {"phi_gc": ores.phi_gc, "radius": ores.radius, "phi_approx": ores.phi_approx, "k": ores.k,
           "quotient_edges": int(oq.col.size)}
    out.update({f: int(ocl.stats[f]) for f in ("stages", "steps", "doublings", "delta_end", "guard_exits",
                                                "node_updates", "centers_drawn")})
    return out


def test_served_results_equal_oracle(env):
    # 24 queries, every graph of the arena at least once, on both lanes: the three largest graphs go to the
    # one-graph lane (big_nodes), the rest to the persistent serving CTAs; every field equals the oracle's
    cd, arena, ids, taus, ns = env
    big = sorted(ns)[-3]
    srv = cd.server_create(arena, ctas=8, big_nodes=big - 1, idle_seconds=2.0)
    rng = np.random.default_rng(9)
    picks = list(range(len(ids))) + [int(x) for x in rng.integers(0, len(ids), 6)]
    seeds = [int(x) for x in rng.integers(1, 1 << 30, len(picks))]
    tickets = [srv.submit(ids[g], taus[g], s) for g, s in zip(picks, seeds)]
    got = {}
    t0 = time.time()
    while len(got) < len(tickets) and time.time() - t0 < 60:
        for t in tickets:
            if t not in got:
                r = srv.poll(t)
                if r is not None:
                    got[t] = r
    srv.free()
    assert len(got) == len(tickets)
    assert sum(ns[g] >= big for g in picks) >= 3 and sum(ns[g] < big for g in picks) >= 3  # both lanes
    for g, s, t in zip(picks, seeds, tickets):
        assert {f: got[t][f] for f in ORACLE_FIELDS} == oracle_result(EDGES[g], taus[g], s), (g, s)


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
