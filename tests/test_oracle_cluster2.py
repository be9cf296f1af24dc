"""Pin the oracle's CLUSTER2 (Algorithm 2, Section 4).

The oracle follows Algorithm 2 literally: an explicit contracted edge list G_i,
PartialGrowth2 as synchronous growing steps to a fixed point, Contract2's
rescaled weights d_u + w - 2 R_CL.  It is pinned against:
  * a restatement with global offsets instead of contractions: a center drawn in
    iteration i starts at g = (i - 1) 2 R_CL, every covered node keeps the g it
    was reached with, and iteration i is one multi-source Dijkstra over the
    uncovered nodes (lexicographic (g, center) keys, edges of weight <= 2 R_CL)
    that keeps the nodes with g <= i 2 R_CL.  Rescaling by 2 R_CL per contraction
    and offsetting the sources by the same amount give the same states, so the
    two must agree exactly on center and D = g_v - g_{c_v};
  * invariants: every node covered, centers self-centred, D_v >= dist_G(c_v, v),
    and every non-center v has a neighbour u of its own cluster with
    D_u + w(u, v) = D_v (D is the length of a path the growth followed);
  * R_CL = 0 (CLUSTER returns singletons): CLUSTER2 draws every node as its own
    center, D = 0;
  * the estimate over CLUSTER2's clustering stays conservative, Phi_approx >= Phi(G).
"""
import heapq

import numpy as np
import pytest

import inputs
import oracle

csgraph = pytest.importorskip("scipy.sparse.csgraph")
sp = pytest.importorskip("scipy.sparse")


def random_graph(seed, n=None, W=100):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(200, 1500))
    m = int(rng.integers(n, 4 * n))
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    w = rng.integers(1, W + 1, m).astype(np.uint32)
    return oracle.build_csr(n, src, dst, w, lcc=True)


def iterations(n):
    L = 1
    while (1 << L) < n:
        L += 1
    return L


def cluster2_offsets(g, tau, seed, d0):
    """Algorithm 2 restated with global offsets (see the module docstring)."""
    R = int(oracle.cluster(g, tau, seed, d0).D.max())
    delta = 2 * R
    n = g.n
    off, col, wt = g.off.astype(np.int64), g.col.astype(np.int64), g.wt.astype(np.int64)
    covered = np.zeros(n, bool)
    center = np.full(n, -1, np.int64)
    gval = np.zeros(n, np.int64)
    for i in range(1, iterations(n) + 1):
        thr = 1 << 32 if (1 << i) >= n else (1 << (32 + i)) // n
        for v in range(n):
            if not covered[v] and int(oracle.philox4x32_10(seed, [v, i, 1, 0])[0]) < thr:
                covered[v] = True
                center[v] = v
                gval[v] = (i - 1) * delta
        limit = i * delta
        best = {}
        heap = []
        for u in np.nonzero(covered)[0]:
            for j in range(off[u], off[u + 1]):
                x, w = col[j], wt[j]
                if covered[x] or w > delta or gval[u] + w > limit:
                    continue
                heapq.heappush(heap, (int(gval[u] + w), int(center[u]), int(x)))
        done = {}
        while heap:
            gx, cx, x = heapq.heappop(heap)
            if x in done:
                continue
            done[x] = (gx, cx)
            for j in range(off[x], off[x + 1]):
                y, w = col[j], wt[j]
                if covered[y] or y in done or w > delta or gx + w > limit:
                    continue
                heapq.heappush(heap, (int(gx + w), cx, int(y)))
        for x, (gx, cx) in done.items():
            covered[x] = True
            center[x] = cx
            gval[x] = gx
        del best
    assert covered.all()
    return center.astype(np.uint32), (gval - gval[center]).astype(np.uint64)


@pytest.mark.parametrize("seed", range(6))
def test_against_offset_restatement_random(seed):
    g = random_graph(seed)
    d0 = oracle.delta0(g)
    for tau in (0.5, 1.0):
        c2 = oracle.cluster2(g, tau, seed, d0)
        center, D = cluster2_offsets(g, tau, seed, d0)
        assert np.array_equal(c2.center, center), tau
        assert np.array_equal(c2.D, D), tau


@pytest.mark.parametrize("e,tau", [(lambda: inputs.grid(24, 100, 1), 0.3),
                                   (lambda: inputs.road_mesh(24, 1000, 3), 0.3),
                                   (lambda: inputs.rmat(9, 8, 1000, 3), 0.5)])
def test_against_offset_restatement_workload_shapes(e, tau):
    el = e()
    g = oracle.build_csr(el.n, el.src, el.dst, el.w, lcc=True)
    d0 = oracle.delta0(g)
    c2 = oracle.cluster2(g, tau, 5, d0)
    center, D = cluster2_offsets(g, tau, 5, d0)
    assert np.array_equal(c2.center, center)
    assert np.array_equal(c2.D, D)
    assert len(np.unique(c2.center)) > 1  # a case with real growth across iterations


def cycle_with_chords(seed, n=2000, chords=20, heavy=0.0):
    # long cycle, few chords: CLUSTER's radius is far below the diameter, so CLUSTER2's clusters keep
    # growing over many iterations through Contract2's rescaled edges; `heavy` of the edges weigh
    # 200..1000, mostly above 2 R_CL (edges CLUSTER2 must never use)
    rng = np.random.default_rng(seed)
    src = np.concatenate([np.arange(n), rng.integers(0, n, chords)]).astype(np.uint32)
    dst = np.concatenate([(np.arange(n) + 1) % n, rng.integers(0, n, chords)]).astype(np.uint32)
    w = rng.integers(1, 11, src.size).astype(np.uint32)
    hv = rng.random(src.size) < heavy
    w[hv] = rng.integers(200, 1001, int(hv.sum())).astype(np.uint32)
    return oracle.build_csr(n, src, dst, w, lcc=True)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("tau", [1.0, 4.0])
@pytest.mark.parametrize("heavy", [0.0, 0.05])
def test_against_offset_restatement_multi_iteration_growth(seed, tau, heavy):
    g = cycle_with_chords(seed, heavy=heavy)
    d0 = oracle.delta0(g)
    c2 = oracle.cluster2(g, tau, seed, d0)
    center, D = cluster2_offsets(g, tau, seed, d0)
    assert np.array_equal(c2.center, center)
    assert np.array_equal(c2.D, D)
    # many nodes were reached one or more iterations after their center was drawn
    assert (c2.D >= 2 * c2.stats["r_cl"]).sum() > g.n // 20


def to_scipy(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.off).astype(np.int64))
    return sp.csr_matrix((g.wt.astype(np.float64), (rows, g.col.astype(np.int64))), shape=(g.n, g.n))


@pytest.mark.parametrize("seed", range(4))
def test_invariants(seed):
    g = random_graph(100 + seed, W=1000) if seed % 2 else cycle_with_chords(seed, n=1500)
    d0 = oracle.delta0(g)
    c2 = oracle.cluster2(g, 0.5, seed, d0)
    center, D = c2.center.astype(np.int64), c2.D.astype(np.int64)
    assert (center >= 0).all() and (center < g.n).all()
    assert (center[center] == center).all() and (D[center] == 0).all()
    dist = csgraph.dijkstra(to_scipy(g), directed=False, indices=np.unique(center))
    row = {c: r for r, c in enumerate(np.unique(center))}
    for v in range(g.n):
        assert D[v] >= dist[row[center[v]], v]
        if center[v] == v:
            continue
        nb = g.col[g.off[v]:g.off[v + 1]].astype(np.int64)
        ww = g.wt[g.off[v]:g.off[v + 1]].astype(np.int64)
        ok = (center[nb] == center[v]) & (D[nb] + ww == D[v])
        assert ok.any(), v
    # radius bound of the literal algorithm: a node reached in iteration i_v by a center of
    # iteration i_c lies within (i_v - i_c + 1) 2 R_CL <= L 2 R_CL
    assert D.max() <= iterations(g.n) * 2 * c2.stats["r_cl"]


def test_singletons_when_cluster_has_radius_zero():
    # 8 tau log n > n: CLUSTER runs no stage, R_CL = 0, so nothing can grow
    g = random_graph(7, n=300)
    c2 = oracle.cluster2(g, 50.0, 3, oracle.delta0(g))
    assert c2.stats["r_cl"] == 0
    assert np.array_equal(c2.center, np.arange(g.n, dtype=np.uint32))
    assert (c2.D == 0).all()
    assert c2.stats["centers_drawn"] == g.n


@pytest.mark.parametrize("seed", range(3))
def test_estimate_is_conservative(seed):
    g = random_graph(200 + seed, W=50)
    c2 = oracle.cluster2(g, 0.5, seed, oracle.delta0(g))
    q = oracle.quotient(g, c2)
    r = oracle.estimate(q, c2)
    d = csgraph.shortest_path(to_scipy(g), method="D", directed=False)
    assert r.phi_approx >= int(d[np.isfinite(d)].max())
