"""Pin the oracle's CLUSTER (Algorithm 1), quotient and estimate (Section 4).

CLUSTER's trajectory is random (Philox draws) and the paper prints no worked
example, so it is pinned by what the paper and the mathematics fix:
  * coverage, self-centred centers, D_v >= dist_G(c_v, v) (Section 3: d_u is an
    upper bound on the distance to the center), D_v <= sum of the stages' Delta;
  * every stage covers at least half of its uncovered nodes or stops at a true
    fixed point, hence at most floor(log2(n / (8 tau log n))) + 1 stages on a
    connected graph (Section 3, "at most O(log n) stages");
  * the conservative estimate Phi_approx >= Phi(G) (Section 4);
  * the special case that reduces to exact APSP: no stage runs
    (|U| < 8 tau log n) -> all clusters are singletons, G_C = G and
    Phi_approx = Phi(G) exactly (p >= 1 cannot occur: the outer test caps
    p = gamma tau log n / |U| at gamma / 8 < 1);
  * closed-form diameters (tests/golden/closed_forms.json);
  * quotient rebuilt independently from the clustering; APSP / SSSP against scipy.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from tests.golden import closed_forms

csgraph = pytest.importorskip("scipy.sparse.csgraph")
sp = pytest.importorskip("scipy.sparse")


def to_scipy(g, w=None):
    rows = np.repeat(np.arange(g.n), np.diff(g.off).astype(np.int64))
    return sp.csr_matrix(((g.wt if w is None else w).astype(np.float64), (rows, g.col.astype(np.int64))),
                         shape=(g.n, g.n))


def exact_diameter(g):
    d = csgraph.shortest_path(to_scipy(g), method="D", directed=False)
    return int(d[np.isfinite(d)].max()) if d.size else 0


def random_graph(seed, n=None):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(20, 200))
    m = int(rng.integers(n, 4 * n))
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    w = rng.integers(1, 50, m).astype(np.uint32)
    return oracle.build_csr(n, src, dst, w, lcc=True)


def check_invariants(g, tau, seed, mode=oracle.DELTA0_AVG):
    d0 = oracle.delta0(g, mode)
    cl = oracle.cluster(g, tau, seed, d0)
    c, D = cl.center.astype(np.int64), cl.D.astype(np.int64)
    assert (c < g.n).all()                                   # every node covered
    assert (c[c] == c).all()                                 # centers are their own center
    assert (D[c] == 0).all()                                 # ... at distance 0
    # D is an upper bound on the true distance to the center
    centers = np.unique(c)
    dist = csgraph.dijkstra(to_scipy(g), directed=False, indices=centers)
    row = {int(x): i for i, x in enumerate(centers)}
    true = dist[[row[int(x)] for x in c], np.arange(g.n)]
    assert (D >= true).all()
    # stage bound on D, from the trace's per-stage final Delta
    fin = cl.trace[cl.trace["kind"] == oracle.TRACE_FINALIZE]
    assert len(fin) == cl.stats["stages"]
    assert D.max() <= int(fin["delta"].astype(np.int64).sum())
    # ... and stage by stage: a node frozen in stage s has D <= Delta_1 + ... + Delta_s (its d is within
    # Delta_s, and R_prev of its cluster within the earlier stages' sum); fin["b"] = the stage's largest D
    assert (fin["b"].astype(np.int64) <= np.cumsum(fin["delta"].astype(np.int64))).all()
    # each stage reaches half coverage or stops at a true fixed point
    tr = cl.trace
    starts = np.flatnonzero(tr["kind"] == oracle.TRACE_STAGE)
    for s in starts:
        U = int(tr["a"][s])
        j = s + 1
        last_cov, guard = None, False
        while j < len(tr) and tr["kind"][j] != oracle.TRACE_FINALIZE:
            if tr["kind"][j] == oracle.TRACE_STEP:
                last_cov = int(tr["b"][j])
            if tr["kind"][j] == oracle.TRACE_GUARD:
                guard = True
            j += 1
        assert guard or 2 * last_cov >= U
    # Delta only doubles and ends where the trace says
    deltas = tr["delta"].astype(np.int64)
    if len(deltas):
        assert (np.diff(deltas) >= 0).all() and cl.stats["delta_end"] == deltas[-1]
    if cl.stats["guard_exits"] == 0 and g.n > 1:
        L = math.log2(g.n)
        bound = math.floor(math.log2(g.n / (8 * tau * L))) + 1 if g.n >= 8 * tau * L else 0
        assert cl.stats["stages"] <= bound
    return cl


@pytest.mark.parametrize("seed", range(12))
def test_invariants_random(seed):
    g = random_graph(seed)
    for tau in (0.05, 0.2, 1.0):
        check_invariants(g, tau, seed)
    check_invariants(g, 0.1, seed, oracle.DELTA0_MIN)


def test_invariants_workload_shapes():
    for e, tau in [(inputs.grid(32, 100, 1), 0.3), (inputs.rmat(10, 8, 1000, 3), 1.0),
                   (inputs.road_mesh(40, 1000, 3), 0.5)]:
        g = oracle.build_csr(e.n, e.src, e.dst, e.w)
        check_invariants(g, tau, 5)


@pytest.mark.parametrize("seed", range(10))
def test_conservative_estimate(seed):
    g = random_graph(50 + seed)
    r, cl, q = oracle.cldiam(g, 0.1, seed)
    phi = exact_diameter(g)
    assert r.phi_approx >= phi
    lb, e0 = oracle.lower_bound(g, oracle.sssp_source(seed, g.n))
    assert e0 <= lb <= phi <= 2 * e0


@pytest.mark.parametrize("seed", range(6))
def test_no_stage_gives_exact_diameter(seed):
    g = random_graph(80 + seed)
    tau = g.n  # 8 tau log n > n: the outer loop never runs, all singletons
    r, cl, q = oracle.cldiam(g, tau, seed)
    assert r.k == g.n and r.radius == 0 and cl.stats["stages"] == 0
    assert r.phi_approx == exact_diameter(g)


def oracle_gamma():
    return 4 * math.log(2)


def test_closed_forms():
    for name, n, s, d, w, diam in closed_forms.load():
        g = oracle.build_csr(n, s, d, w, lcc=True)
        assert exact_diameter(g) == diam, name
        r, _, _ = oracle.cldiam(g, float(n), 1)          # all singletons: exact
        assert r.phi_approx == diam, name
        r, _, _ = oracle.cldiam(g, 0.05, 1)               # real clustering: conservative
        assert r.phi_approx >= diam, name
        lb, e0 = oracle.lower_bound(g, oracle.sssp_source(1, g.n))
        assert lb <= diam <= 2 * e0, name


def ref_quotient(g, center, D):
    centers = sorted(set(int(x) for x in center))
    rank = {c: i for i, c in enumerate(centers)}
    cid = np.array([rank[int(c)] for c in center], np.uint32)
    best = {}
    for u in range(g.n):
        for j in range(int(g.off[u]), int(g.off[u + 1])):
            v = int(g.col[j])
            a, b = int(cid[u]), int(cid[v])
            if a == b:
                continue
            wq = int(D[u]) + int(g.wt[j]) + int(D[v])
            best[(a, b)] = min(best.get((a, b), wq), wq)
    return len(centers), cid, best


@pytest.mark.parametrize("seed", range(8))
def test_quotient_and_apsp(seed):
    g = random_graph(200 + seed)
    cl = oracle.cluster(g, 0.1, seed, oracle.delta0(g))
    q = oracle.quotient(g, cl)
    k, cid, best = ref_quotient(g, cl.center, cl.D)
    assert q.k == k and np.array_equal(q.cid, cid)
    got = {}
    for a in range(q.k):
        cols = q.col[int(q.off[a]):int(q.off[a + 1])]
        assert (np.diff(cols.astype(np.int64)) > 0).all()     # sorted, unique
        for j in range(int(q.off[a]), int(q.off[a + 1])):
            got[(a, int(q.col[j]))] = int(q.w[j])
    assert got == best
    assert all(got[(b, a)] == x for (a, b), x in got.items())  # symmetric
    # Phi(G_C) against scipy
    rows = np.repeat(np.arange(q.k), np.diff(q.off).astype(np.int64))
    M = sp.csr_matrix((q.w.astype(np.float64), (rows, q.col.astype(np.int64))), shape=(q.k, q.k))
    d = csgraph.shortest_path(M, method="D", directed=False)
    assert oracle.apsp_max(q) == int(d[np.isfinite(d)].max())


@pytest.mark.parametrize("seed", range(6))
def test_dijkstra_against_scipy(seed):
    g = random_graph(300 + seed)
    s = oracle.sssp_source(seed, g.n)
    got = oracle.dijkstra(g, s)
    ref = csgraph.dijkstra(to_scipy(g), directed=False, indices=s)
    assert np.array_equal(got.astype(np.float64), ref)


def test_determinism_and_seed_dependence():
    e = inputs.grid(32, 100, 1)
    g = oracle.build_csr(e.n, e.src, e.dst, e.w)
    a = oracle.cluster(g, 0.3, 11, oracle.delta0(g))
    b = oracle.cluster(g, 0.3, 11, oracle.delta0(g))
    c = oracle.cluster(g, 0.3, 12, oracle.delta0(g))
    assert np.array_equal(a.center, b.center) and np.array_equal(a.D, b.D)
    assert not np.array_equal(a.center, c.center)


def test_center_draw_rule():
    # stage-1 centers are exactly the nodes whose Philox(seed; v, 1) word 0 is below thr
    e = inputs.grid(16, 10, 2)
    g = oracle.build_csr(e.n, e.src, e.dst, e.w)
    tau, seed = 0.5, 9
    cl = oracle.cluster(g, tau, seed, oracle.delta0(g))
    L = math.log2(g.n)
    p = oracle_gamma() * tau * L / g.n
    thr = math.floor(p * 2 ** 32)
    drawn = [v for v in range(g.n) if int(oracle.philox4x32_10(seed, [v, 1, 0, 0])[0]) < thr]
    st = cl.trace[cl.trace["kind"] == oracle.TRACE_STAGE][0]
    assert int(st["b"]) == len(drawn)
    for v in drawn:   # a stage-1 center keeps itself
        assert int(cl.center[v]) == v
