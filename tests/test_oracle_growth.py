"""Pin the Delta-growing step of Section 3 (and PartialGrowth's fixed point).

Characterisation used (independent of the oracle's loop): after t synchronous
steps, each unfrozen node holds the lexicographic minimum of (distance, center)
over its start key and all walks of at most t edges that
  * start at a frozen node u with key (0, c_u)  (Procedure Contract: u stands
    for its contracted center), or at an unfrozen node with a key (d, c),
  * pass only through unfrozen nodes, and
  * keep every prefix length <= Delta (the step's d_u + w <= Delta test).
At the fixed point ("no state is updated", PartialGrowth) the same minimum
over walks of any length equals a multi-source Dijkstra on (distance, center)
keys.  Both are computed here by brute force.
"""
import heapq

import numpy as np
import pytest

import oracle

INF = oracle.INF_KEY


def tiny_graph(rng):
    n = int(rng.integers(2, 8))
    edges = {}
    for _ in range(int(rng.integers(1, 2 * n + 2))):
        a, b = (int(x) for x in rng.integers(0, n, 2))
        if a != b:
            edges[(min(a, b), max(a, b))] = int(rng.integers(1, 7))
    src = np.array([e[0] for e in edges], np.uint32)
    dst = np.array([e[1] for e in edges], np.uint32)
    w = np.array(list(edges.values()), np.uint32)
    return oracle.build_csr(n, src, dst, w, lcc=False)


def adj(g):
    out = {u: [] for u in range(g.n)}
    for u in range(g.n):
        for j in range(int(g.off[u]), int(g.off[u + 1])):
            out[u].append((int(g.col[j]), int(g.wt[j])))
    return out


def random_state(rng, g, delta):
    frozen = (rng.random(g.n) < 0.3).astype(np.uint8)
    center = np.full(g.n, oracle.NONE, np.uint32)
    key = np.full(g.n, INF, np.uint64)
    for v in range(g.n):
        if frozen[v]:
            center[v] = int(rng.integers(0, g.n))
        else:
            r = rng.random()
            if r < 0.3:
                key[v] = v                              # a fresh center: (0, v)
            elif r < 0.5:
                d = int(rng.integers(0, delta + 1))
                key[v] = (d << 32) | int(rng.integers(0, g.n))
    return key, frozen, center


def brute_walks(g, key, frozen, center, delta, t, D=None):
    # D given: cumulative contract mode, a frozen start u has length D_u (and relaxes only if D_u < Delta)
    A = adj(g)
    best = [int(key[v]) if not frozen[v] else None for v in range(g.n)]
    starts = []
    for s in range(g.n):
        if frozen[s]:
            if D is None:
                starts.append((s, 0, int(center[s])))
            elif int(D[s]) < delta:
                starts.append((s, int(D[s]), int(center[s])))
        elif int(key[s]) != INF:
            starts.append((s, int(key[s]) >> 32, int(key[s]) & 0xFFFFFFFF))

    def walk(x, length, c, hops):
        if hops == t:
            return
        for (v, w) in A[x]:
            if frozen[v] or length + w > delta:
                continue
            k = ((length + w) << 32) | c
            if k < best[v]:
                best[v] = k
            walk(v, length + w, c, hops + 1)

    for (s, d, c) in starts:
        walk(s, d, c, 0)
    return best


def lex_dijkstra(g, key, frozen, center, delta):
    A = adj(g)
    best = {v: int(key[v]) for v in range(g.n) if not frozen[v]}
    h = []
    for s in range(g.n):
        if frozen[s]:
            h.append((0, int(center[s]), s, True))
        elif int(key[s]) != INF:
            h.append((int(key[s]) >> 32, int(key[s]) & 0xFFFFFFFF, s, False))
    heapq.heapify(h)
    done = set()
    while h:
        d, c, x, is_frozen = heapq.heappop(h)
        tag = (x, is_frozen)
        if tag in done:
            continue
        if not is_frozen and ((d << 32) | c) != best[x]:
            continue
        done.add(tag)
        for (v, w) in A[x]:
            if frozen[v] or d + w > delta:
                continue
            k = ((d + w) << 32) | c
            if k < best[v]:
                best[v] = k
                heapq.heappush(h, (d + w, c, v, False))
    return best


@pytest.mark.parametrize("seed", range(40))
def test_t_steps_equal_bounded_walks(seed):
    rng = np.random.default_rng(seed)
    g = tiny_graph(rng)
    delta = int(rng.integers(1, 13))
    key, frozen, center = random_state(rng, g, delta)
    prev = [int(x) for x in key]
    for t in range(1, 5):
        got, upd = oracle.growth_steps(g, key, frozen, center, delta, t)
        ref = brute_walks(g, key, frozen, center, delta, t)
        for v in range(g.n):
            if not frozen[v]:
                assert int(got[v]) == ref[v], (seed, t, v)
        # the last step's update count = nodes whose minimum improved with the t-th hop
        ref_prev = brute_walks(g, key, frozen, center, delta, t - 1) if t > 1 else prev
        changed = sum(1 for v in range(g.n) if not frozen[v] and ref[v] < ref_prev[v])
        assert int(upd[-1]) == changed


@pytest.mark.parametrize("seed", range(40))
def test_cumulative_steps_equal_bounded_walks(seed):
    # cumulative contract mode: a frozen node starts its walks at its own bound D_u instead of 0
    rng = np.random.default_rng(500 + seed)
    g = tiny_graph(rng)
    delta = int(rng.integers(1, 13))
    key, frozen, center = random_state(rng, g, delta)
    D = np.where(frozen != 0, rng.integers(0, delta + 3, g.n), 0).astype(np.uint64)
    prev = [int(x) for x in key]
    for t in range(1, 5):
        got, upd = oracle.growth_steps(g, key, frozen, center, delta, t, D=D)
        ref = brute_walks(g, key, frozen, center, delta, t, D=D)
        for v in range(g.n):
            if not frozen[v]:
                assert int(got[v]) == ref[v], (seed, t, v)
        ref_prev = brute_walks(g, key, frozen, center, delta, t - 1, D=D) if t > 1 else prev
        changed = sum(1 for v in range(g.n) if not frozen[v] and ref[v] < ref_prev[v])
        assert int(upd[-1]) == changed
    # all frozen bounds at 0 give the default mode's steps
    got0, _ = oracle.growth_steps(g, key, frozen, center, delta, 3, D=np.zeros(g.n, np.uint64))
    got1, _ = oracle.growth_steps(g, key, frozen, center, delta, 3)
    assert np.array_equal(got0, got1)


@pytest.mark.parametrize("seed", range(40))
def test_fixed_point_equals_lexicographic_dijkstra(seed):
    rng = np.random.default_rng(100 + seed)
    g = tiny_graph(rng)
    delta = int(rng.integers(1, 20))
    key, frozen, center = random_state(rng, g, delta)
    got, upd = oracle.growth_steps(g, key, frozen, center, delta, g.n + 2)
    assert upd[-1] == 0  # n+1 steps always reach the fixed point on n nodes
    ref = lex_dijkstra(g, key, frozen, center, delta)
    for v, k in ref.items():
        assert int(got[v]) == k, (seed, v)


def test_tie_break_smallest_center():
    # two centers at equal distance from node 1: the smaller center id must win
    g = oracle.build_csr(3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([5, 5], np.uint32),
                         lcc=False)
    key = np.array([0 | 0, INF, (0 << 32) | 2], np.uint64)
    got, _ = oracle.growth_steps(g, key, np.zeros(3, np.uint8), np.full(3, oracle.NONE, np.uint32), 10, 1)
    assert int(got[1]) == (5 << 32) | 0
    # the relaxer condition d_u < Delta: a node sitting exactly at Delta does not relax
    key = np.array([(4 << 32) | 0, INF, INF], np.uint64)
    got, _ = oracle.growth_steps(g, key, np.zeros(3, np.uint8), np.full(3, oracle.NONE, np.uint32), 9, 3)
    assert int(got[1]) == (9 << 32) | 0 and int(got[2]) == INF
