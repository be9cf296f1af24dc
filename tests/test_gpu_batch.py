"""Many-graph form (one persistent launch) against the one-graph path and the oracle.

Every batched result must equal cldiam_cluster + cldiam_quotient_build +
cldiam_estimate on the same graph, tau and seed (integers: bit-exact).
"""
import math

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


def oracle_result(e, tau, seed):
    """The whole method on the CPU oracle, as a dict over ORACLE_FIELDS."""
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    ores, ocl, oq = oracle.cldiam(og, tau, seed)
    out = {"phi_gc": ores.phi_gc, "radius": ores.radius, "phi_approx": ores.phi_approx, "k": ores.k,
           "quotient_edges": int(oq.col.size)}
    out.update({f: int(ocl.stats[f]) for f in ("stages", "steps", "doublings", "delta_end", "guard_exits",
                                                "node_updates", "centers_drawn")})
    return out


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    return m


def tau_for(n):
    # about sqrt(n) clusters: each stage draws ~gamma tau log n centers, about log2(n)/2 stages
    L = max(1.0, math.log2(max(n, 2)))
    return max(0.05, math.sqrt(n) / (4 * math.log(2) * L * max(1.0, L / 2)))


def plain(cd, g, tau, seed, mode=0):
    c = cd.cluster(g, tau, seed, delta0_mode=mode)
    return cd.estimate(cd.quotient_build(c))


def test_mixture_matches_one_graph_path(cd):
    arena = cd.arena_create()
    graphs = []
    for gi in range(24):
        kind, scale, side, sub = inputs.mix_params(4, gi)
        e = inputs.rmat(min(scale, 12), 8, 1000, sub) if kind == 0 else inputs.grid(min(side, 96), 1000, sub)
        gid = arena.add(e.src, e.dst, e.w, e.n)
        graphs.append((gid, e))
    ids = [gid for gid, _ in graphs]
    taus = [tau_for(arena.graph(gid).n) for gid in ids]
    seeds = [1000 + i for i in range(len(ids))]
    res, st = arena.run(ids, taus, seeds)
    assert all(x == 0 for x in st)
    for (gid, e), tau, seed, r in zip(graphs, taus, seeds, res):
        ref = plain(cd, arena.graph(gid), tau, seed)
        assert {f: r[f] for f in FIELDS} == {f: ref[f] for f in FIELDS}, (gid, e)
    # every graph against the oracle, every field it defines
    for (gid, e), tau, seed, r in zip(graphs, taus, seeds, res):
        assert {f: r[f] for f in ORACLE_FIELDS} == oracle_result(e, tau, seed), (gid, e.n)


def test_repeated_jobs_and_edge_cases(cd):
    arena = cd.arena_create()
    z = np.zeros(0, np.uint32)
    g_single = arena.add(z, z, z, 1)
    n, rng = 300, np.random.default_rng(3)
    s = rng.integers(0, n, 200).astype(np.uint32); d = rng.integers(0, n, 200).astype(np.uint32)
    w = rng.integers(1, 50, 200).astype(np.uint32)
    g_disc = arena.add(s, d, w, n, lcc=False)            # disconnected: fixed-point guard path
    e = inputs.grid(128, 100, 9)
    g_big_k = arena.add(e.src, e.dst, e.w, e.n)          # tau huge: all singletons, k = 16384 > dense capacity
    e2 = inputs.rmat(11, 8, 1 << 20, 5)
    g_r = arena.add(e2.src, e2.dst, e2.w, e2.n)
    ids = [g_single, g_disc, g_big_k, g_r, g_r, g_disc]
    taus = [1.0, 0.2, 1e7, 0.7, 0.7, 0.05]
    seeds = [1, 2, 3, 4, 4, 9]
    res, st = arena.run(ids, taus, seeds)
    assert all(x == 0 for x in st)
    for gid, tau, seed, r in zip(ids, taus, seeds, res):
        ref = plain(cd, arena.graph(gid), tau, seed)
        assert {f: r[f] for f in FIELDS} == {f: ref[f] for f in FIELDS}, gid
    assert res[2]["k"] == 16384 and res[3] == res[4]


def test_budget_admission(cd):
    arena = cd.arena_create(hbm_budget_bytes=1 << 20)
    e = inputs.grid(200, 100, 1)   # ~1.9 MB of CSR: over a 1 MiB budget
    with pytest.raises(cd.CldiamError) as ei:
        arena.add(e.src, e.dst, e.w, e.n)
    assert ei.value.status == -2


@pytest.fixture(scope="module")
def split_arena(cd):
    """Graphs large enough to outweigh the per-CTA average of a small batch (they run on the one-graph
    path first), a large disconnected one (no LCC), and small ones (the persistent launch)."""
    arena = cd.arena_create()
    big = [inputs.rmat(16, 16, 1000, 21), inputs.grid(400, 1000, 22), inputs.road_mesh(512, 1000, 23)]
    rng = np.random.default_rng(24)
    n = 200_000
    disc = inputs.EdgeList(n, rng.integers(0, n, 160_000).astype(np.uint32),
                           rng.integers(0, n, 160_000).astype(np.uint32),
                           rng.integers(1, 1000, 160_000).astype(np.uint32))
    small = [inputs.rmat(10, 8, 1000, 25), inputs.grid(30, 1000, 26)]
    graphs = [(arena.add(e.src, e.dst, e.w, e.n), e) for e in big + small]
    graphs.append((arena.add(disc.src, disc.dst, disc.w, disc.n, lcc=False), disc))
    return arena, graphs


@pytest.mark.parametrize("split", [1, 2])
def test_split_batches_match_one_graph_path(cd, split_arena, split):
    arena, graphs = split_arena
    ids = [gid for gid, _ in graphs] + [graphs[0][0]]
    taus = [tau_for(arena.graph(gid).n) for gid in ids]
    taus[-1] *= 30  # R-MAT 16 with k ~ 2,000: above the kernel's dense quotient capacity when in the launch
    seeds = [40 + i for i in range(len(ids))]
    cd.tuning_set(batch_split=split)
    try:
        for mode, cap in ((cd.CONTRACT_RESET, 0), (cd.CONTRACT_CUMULATIVE, 3)):
            res, st = arena.run(ids, taus, seeds, contract_mode=mode, step_cap=cap)
            assert all(x == 0 for x in st)
            for gid, tau, seed, r in zip(ids, taus, seeds, res):
                c = cd.cluster(arena.graph(gid), tau, seed, contract_mode=mode, step_cap=cap)
                ref = cd.estimate(cd.quotient_build(c))
                assert {f: r[f] for f in FIELDS} == {f: ref[f] for f in FIELDS}, (gid, mode)
            start, end = arena.job_times(len(ids))
            assert np.all(end >= start) and start.min() == 0.0
    finally:
        cd.tuning_set()


def test_split_batch_matches_oracle(cd, split_arena):
    arena, graphs = split_arena
    ids = [gid for gid, _ in graphs]
    taus = [tau_for(arena.graph(gid).n) for gid in ids]
    seeds = [70 + i for i in range(len(ids))]
    res, st = arena.run(ids, taus, seeds)
    assert all(x == 0 for x in st)
    for (gid, e), tau, seed, r in zip(graphs, taus, seeds, res):
        if gid == graphs[-1][0]:  # no LCC: the oracle's CSR without it
            og = oracle.build_csr(e.n, e.src, e.dst, e.w, lcc=False)
            ores, ocl, oq = oracle.cldiam(og, tau, seed)
            assert (r["k"], r["phi_gc"], r["phi_approx"], r["stages"]) == (ores.k, ores.phi_gc, ores.phi_approx,
                                                                           ocl.stats["stages"])
        else:
            assert {f: r[f] for f in ORACLE_FIELDS} == oracle_result(e, tau, seed), (gid, e.n)
