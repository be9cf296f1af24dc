"""The two forms of a Delta-growing step (Section 3) against the oracle: the pushed form (each
relaxer lowers its neighbours' keys) and the dense pull form (each unfrozen node takes the
smallest candidate over its own adjacency, read from the start-of-step keys).  Which form runs is
a tuning knob; both must give exactly the oracle's synchronous steps, in both contract modes and
with the growing-step cap.

Integers: bit-exact (centers, D, cluster ids, counters, quotient CSR, estimate).
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

# pull_ratio -1: never dense, 1e-9: dense at every step, default: switching by the relaxers' share
FORMS = {"push": {"pull_ratio": -1.0}, "pull": {"pull_ratio": 1e-9}, "mixed": {}}


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    yield m
    m.tuning_set()


def graphs():
    out = [inputs.grid(24, 100, 1), inputs.grid(45, 1000, 2), inputs.road_mesh(64, 1000, 3)]
    for scale, ef, seed in ((9, 8, 4), (12, 8, 5), (14, 16, 6)):
        out.append(inputs.rmat(scale, ef, 1000, seed))
    rng = np.random.default_rng(11)
    n, m = 3000, 9000  # random multigraph with duplicates, self-loops and a hub of degree ~ 2,000
    src = np.concatenate([rng.integers(0, n, m), np.zeros(2000, np.int64)]).astype(np.uint32)
    dst = np.concatenate([rng.integers(0, n, m), rng.integers(1, n, 2000)]).astype(np.uint32)
    w = rng.integers(1, 60, src.size).astype(np.uint32)
    out.append(inputs.EdgeList(n, src, dst, w))
    return out


GRAPHS = graphs()


def check(cd, e, tau, seed, mode=0, cap=0, d0_mode=0):
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    c = cd.cluster(g, tau, seed, delta0_mode=d0_mode, contract_mode=mode, step_cap=cap)
    ocl = oracle.cluster(og, tau, seed, oracle.delta0(og, d0_mode), contract_mode=mode, step_cap=cap)
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
    return r


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_forms_match_oracle(cd, form, gi):
    cd.tuning_set(**FORMS[form])
    e = GRAPHS[gi]
    cd.profile_reset()
    for tau, seed in ((0.3, 1), (2.0, 7)):
        check(cd, e, tau, seed)
    check(cd, e, 0.5, 3, d0_mode=1)  # Delta from the minimum weight: many doublings
    prof = cd.profile_get()
    # queued steps launch both forms and the one not taken returns at once: the work shows in the bytes
    if form == "pull":
        assert prof["relax_pull"]["bytes"] > 0 and prof["relax"]["bytes"] == 0
    elif form == "push":
        assert prof["relax_pull"]["launches"] == 0 and prof["relax"]["bytes"] > 0


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("mode,cap", [(1, 0), (0, 1), (1, 2), (0, 3)])
def test_forms_options(cd, form, mode, cap):
    cd.tuning_set(**FORMS[form])
    for e in (GRAPHS[1], GRAPHS[4], GRAPHS[6]):
        check(cd, e, 0.4, 5, mode=mode, cap=cap)


def test_mixed_forms_switch_midway(cd):
    # the default threshold switches between the forms from step to step: the pushed steps must keep
    # the start-of-step keys that a later dense step reads up to date
    cd.tuning_set()
    for e in GRAPHS:
        for mode in (0, 1):
            check(cd, e, 0.7, 9, mode=mode)
    for ratio in (0.05, 0.2, 0.5, 0.9):
        cd.tuning_set(pull_ratio=ratio)
        check(cd, GRAPHS[5], 1.5, 2)
        check(cd, GRAPHS[2], 0.4, 4, mode=1)


def test_pull_needs_every_row_to_have_an_entry(cd):
    # without the LCC option isolated nodes have no entry; the library keeps the pushed form there
    cd.tuning_set(pull_ratio=1e-9)
    rng = np.random.default_rng(3)
    n = 500
    src = rng.integers(0, 200, 600).astype(np.uint32)
    dst = rng.integers(0, 200, 600).astype(np.uint32)
    w = rng.integers(1, 50, 600).astype(np.uint32)
    g = cd.build_csr(src, dst, w, n, lcc=False)
    og = oracle.build_csr(n, src, dst, w, lcc=False)
    cd.profile_reset()
    c = cd.cluster(g, 0.2, 1)
    ocl = oracle.cluster(og, 0.2, 1, oracle.delta0(og))
    center, D, _ = c.copy()
    assert np.array_equal(center, ocl.center) and np.array_equal(D.astype(np.uint64), ocl.D)
    assert cd.profile_get()["relax_pull"]["bytes"] == 0
    cd.tuning_set()


@pytest.mark.parametrize("seed", range(4))
def test_disconnected_graphs(cd, seed):
    # no LCC: stages that draw no center in a component end at the fixed-point guard
    rng = np.random.default_rng(200 + seed)
    n = 300
    src = rng.integers(0, n, 200).astype(np.uint32)
    dst = rng.integers(0, n, 200).astype(np.uint32)
    w = rng.integers(1, 50, 200).astype(np.uint32)
    g = cd.build_csr(src, dst, w, n, lcc=False)
    og = oracle.build_csr(n, src, dst, w, lcc=False)
    for ratio in (-1.0, 1e-9):
        cd.tuning_set(pull_ratio=ratio)
        c = cd.cluster(g, 0.2, seed)
        ocl = oracle.cluster(og, 0.2, seed, oracle.delta0(og))
        center, D, _ = c.copy()
        assert np.array_equal(center, ocl.center) and np.array_equal(D.astype(np.uint64), ocl.D)
        info = c.info()
        for f in ("stages", "steps", "doublings", "delta_end", "guard_exits", "node_updates", "centers_drawn"):
            assert info[f] == ocl.stats[f], f
    cd.tuning_set()


@pytest.mark.parametrize("which", ["road_mesh_2048", "rmat_16"])
def test_repeated_runs_give_the_same_integers(cd, which):
    # every call is deterministic: repeated runs in both growing-step forms give the same centers, D and counters
    e = inputs.road_mesh(2048, 1000, 3) if which == "road_mesh_2048" else inputs.rmat(16, 16, 1000, 8)
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    tau = 3.0 if which == "road_mesh_2048" else 1.5
    fields = ("stages", "steps", "doublings", "delta_end", "guard_exits", "node_updates", "centers_drawn")
    ref = cd.cluster(g, tau, 3)
    rc, rD, _ = ref.copy()
    rinfo = {f: ref.info()[f] for f in fields}
    try:
        for ratio in (-1.0, 0.3, 1e-9):
            cd.tuning_set(pull_ratio=ratio)
            for it in range(8):
                c = cd.cluster(g, tau, 3)
                center, D, _ = c.copy()
                assert np.array_equal(center, rc) and np.array_equal(D, rD), (ratio, it)
                assert {f: c.info()[f] for f in fields} == rinfo, (ratio, it)
    finally:
        cd.tuning_set()
