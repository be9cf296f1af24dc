"""Tuning knobs on the GPU: every candidate value of every knob gives the same integers as the
defaults (centers, D, quotient CSR, estimate, Delta-stepping distances, many-graph results), and
the autotuners pick a setting, cache it for the size class, and runs that use the cached choice
still agree with the oracle."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

CANDIDATES = {
    "pull_ratio": [-1.0, 0.15, 0.5, 0.8],
    "relax_ctas_per_sm": [2, 4],
    "dense_quotient_k": [1024, 8192],
    "apsp_sources_per_cta": [1, 4, 8],
    "apsp_fw_density": [4, 16],
}


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    m.tuning_set()
    m.tuning_cache_clear()
    yield m
    m.tuning_set()
    m.tuning_cache_clear()


GRAPHS = [inputs.grid(40, 1000, 2), inputs.rmat(12, 8, 1000, 5), inputs.road_mesh(64, 1000, 3)]


def full(cd, g, tau, seed):
    c = cd.cluster(g, tau, seed)
    q = cd.quotient_build(c)
    return c.copy(), q.copy(), cd.estimate(q)


def same(a, b):
    (ca, qa, ra), (cb, qb, rb) = a, b
    return all(np.array_equal(x, y) for x, y in zip(ca + qa, cb + qb)) and ra == rb


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_every_candidate_gives_the_default_result(cd, gi):
    e = GRAPHS[gi]
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    cd.tuning_set()
    for tau, seed in ((0.3, 1), (3.0, 2)):  # ~sqrt(n) clusters, and a large-k quotient (dense paths)
        ref = full(cd, g, tau, seed)
        for knob, values in CANDIDATES.items():
            for v in values:
                cd.tuning_set(**{knob: v})
                assert same(full(cd, g, tau, seed), ref), (knob, v, tau)
    cd.tuning_set()
    src = cd.sssp_source(g, 3)
    dref, eref, _ = cd.sssp_delta(g, src)
    for scale in (2, 4, 8):
        cd.tuning_set(sssp_delta_scale=scale)
        d, ecc, _ = cd.sssp_delta(g, src)
        assert np.array_equal(d, dref) and ecc == eref
    cd.tuning_set()


def test_autotune_graph_caches_and_agrees_with_oracle(cd):
    cd.tuning_set()
    cd.tuning_cache_clear()
    e = inputs.rmat(14, 16, 1 << 20, 2)
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    best = cd.autotune_graph(g, 1.0, 3, reps=2)
    cls = cd.size_class(g.nnz)
    cached = cd.tuning_cache_get(0, cls)
    for k in ("pull_ratio", "relax_ctas_per_sm", "dense_quotient_k", "apsp_sources_per_cta",
              "apsp_fw_density"):
        assert abs(cached[k] - best[k]) < 1e-6, k
    assert cd.tuning_effective(0, cls)["apsp_fw_density"] == best["apsp_fw_density"]
    # a run that takes the cached knobs matches the oracle
    (center, D, cid), _, r = full(cd, g, 1.0, 3)
    ores, ocl, oq = oracle.cldiam(og, 1.0, 3)
    assert np.array_equal(center, ocl.center) and np.array_equal(D.astype(np.uint64), ocl.D)
    assert (r["k"], r["phi_gc"], r["phi_approx"]) == (ores.k, ores.phi_gc, ores.phi_approx)
    # Delta-stepping's bucket width
    src = cd.sssp_source(g, 3)
    bs = cd.autotune_sssp(g, src, reps=2)
    assert bs["sssp_delta_scale"] in (1.0, 2.0, 4.0, 8.0)
    d, _, _ = cd.sssp_delta(g, src)
    assert np.array_equal(d.astype(np.uint64), oracle.dijkstra(og, src))
    cd.tuning_cache_clear()


def test_autotune_batch_and_fw_cutover(cd):
    from inputs.workloads import mixture_tau
    cd.tuning_set()
    cd.tuning_cache_clear()
    arena = cd.arena_create()
    ids = []
    for gi in range(16):
        kind, scale, side, sub = inputs.mix_params(4, gi)
        e = inputs.rmat(min(scale, 11), 8, 1000, sub) if kind == 0 else inputs.grid(min(side, 64), 1000, sub)
        ids.append(arena.add(e.src, e.dst, e.w, e.n))
    taus = [mixture_tau(arena.graph(i).n) for i in ids]
    seeds = [500 + i for i in range(len(ids))]
    ref, st = arena.run(ids, taus, seeds)
    assert all(x == 0 for x in st)
    for fw_k in (1, 64, 128, 200):
        cd.tuning_set(batch_fw_k=fw_k)
        assert arena.run(ids, taus, seeds)[0] == ref, fw_k
    cd.tuning_set()
    best = arena.autotune(ids, taus, seeds, reps=2)
    assert best["batch_fw_k"] in (64, 128, 200) and best["batch_split"] in (1, 2)
    assert arena.run(ids, taus, seeds)[0] == ref
    cd.tuning_cache_clear()
