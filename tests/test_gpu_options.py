"""CLUSTER options on the GPU against the oracle: the cumulative contract mode and the cap on
growing steps per PartialGrowth (end of Section 3), one-graph and many-graph forms.

Integers: bit-exact (centers, D, cluster ids, counters, quotient CSR, estimate).
"""
import math

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

MODES = [(0, 0), (1, 0), (0, 1), (1, 1), (0, 3), (1, 2)]  # (contract_mode, step_cap)


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    return m


def workloads():
    out = []
    for side, W, seed in ((24, 100, 1), (40, 1000, 2)):
        out.append(inputs.grid(side, W, seed))
    out.append(inputs.road_mesh(48, 1000, 3))
    for scale, seed in ((10, 4), (12, 5)):
        out.append(inputs.rmat(scale, 8, 1000, seed))
    return out


WL = workloads()


def check(cd, e, tau, seed, mode, cap, qmode=0):
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    d0 = oracle.delta0(og)
    c = cd.cluster(g, tau, seed, contract_mode=mode, step_cap=cap, quotient_mode=qmode)
    ocl = oracle.cluster(og, tau, seed, d0, contract_mode=mode, step_cap=cap)
    center, D, cid = c.copy()
    assert np.array_equal(center, ocl.center)
    assert np.array_equal(D.astype(np.uint64), ocl.D)
    info = c.info()
    for f in ("stages", "steps", "doublings", "delta_end", "guard_exits", "node_updates", "centers_drawn"):
        assert info[f] == ocl.stats[f], f
    q = cd.quotient_build(c)
    oq = oracle.quotient(og, ocl)
    assert np.array_equal(cid, oq.cid)
    qoff, qcol, qw = q.copy()
    assert np.array_equal(qoff, oq.off) and np.array_equal(qcol, oq.col) and np.array_equal(qw.astype(np.uint64), oq.w)
    r = cd.estimate(q)
    ores = oracle.estimate(oq, ocl)
    assert (r["k"], r["phi_gc"], r["radius"], r["phi_approx"]) == (ores.k, ores.phi_gc, ores.radius, ores.phi_approx)
    if mode == 1:
        assert r["radius"] <= info["delta_end"]  # the cumulative radius bound
    return r


@pytest.mark.parametrize("wi", range(len(WL)))
@pytest.mark.parametrize("mode,cap", MODES)
def test_options_one_graph(cd, wi, mode, cap):
    e = WL[wi]
    for tau, seed in ((0.4, 1), (1.5, 9)):
        check(cd, e, tau, seed, mode, cap)


@pytest.mark.parametrize("seed", range(6))
def test_options_random_graphs(cd, seed):
    rng = np.random.default_rng(40 + seed)
    n = int(rng.integers(50, 600))
    m = int(rng.integers(n, 4 * n))
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    w = rng.integers(1, 200, m).astype(np.uint32)
    e = inputs.EdgeList(n, src, dst, w, name=f"random{seed}")
    for mode, cap in MODES:
        check(cd, e, 0.3 + 0.2 * seed, seed, mode, cap, qmode=seed % 3)


def test_options_many_graph(cd):
    arena = cd.arena_create()
    ids = []
    for e in WL:
        ids.append(arena.add(e.src, e.dst, e.w, e.n))
    taus = [0.4 + 0.1 * i for i in range(len(ids))]
    seeds = [7 + i for i in range(len(ids))]
    for mode, cap in MODES:
        res, st = arena.run(ids, taus, seeds, contract_mode=mode, step_cap=cap)
        assert all(x == 0 for x in st)
        for gid, e, tau, seed, r in zip(ids, WL, taus, seeds, res):
            og = oracle.build_csr(e.n, e.src, e.dst, e.w)
            ocl = oracle.cluster(og, tau, seed, oracle.delta0(og), contract_mode=mode, step_cap=cap)
            ores = oracle.estimate(oracle.quotient(og, ocl), ocl)
            assert (r["k"], r["phi_gc"], r["radius"], r["phi_approx"]) == \
                (ores.k, ores.phi_gc, ores.radius, ores.phi_approx), (gid, mode, cap)
            for f in ("stages", "steps", "doublings", "node_updates"):
                assert r[f] == ocl.stats[f], (gid, mode, cap, f)


def test_unknown_contract_mode_is_rejected(cd):
    e = WL[0]
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    with pytest.raises(cd.CldiamError) as ei:
        cd.cluster(g, 0.5, 1, contract_mode=2)
    assert ei.value.status == -1
