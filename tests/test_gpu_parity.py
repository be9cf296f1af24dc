"""GPU path vs the CPU oracle, element by element (integers: bit-exact).

Every call goes through the C ABI (libcldiam.so via the Python binding).
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    return m


def rand_edges(seed, n=None, m=None, wmax=50, loops=True):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(2, 400))
    m = m if m is not None else int(rng.integers(n // 2, 4 * n))
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    if not loops:
        dst = np.where(src == dst, (dst + 1) % n, dst).astype(np.uint32)
    w = rng.integers(1, wmax + 1, m).astype(np.uint32)
    return n, src, dst, w


def check_csr(cd, n, src, dst, w, lcc):
    g = cd.build_csr(src, dst, w, n, lcc=lcc)
    og = oracle.build_csr(n, src, dst, w, lcc=lcc)
    off, col, ww, orig = g.copy()
    assert g.n == og.n and g.nnz == og.nnz
    assert np.array_equal(off, og.off)
    assert np.array_equal(col, og.col)
    assert np.array_equal(ww, og.wt)
    assert np.array_equal(orig, og.orig)
    return g, og


def check_cluster(cd, g, og, tau, seed, mode=0):
    mode_d0 = mode
    c = cd.cluster(g, tau, seed, delta0_mode=mode)
    d0 = oracle.delta0(og, mode)
    assert g.delta0(mode) == d0
    ocl = oracle.cluster(og, tau, seed, d0)
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
    assert q.info()[0] == oq.k
    assert np.array_equal(qoff, oq.off)
    assert np.array_equal(qcol, oq.col)
    assert np.array_equal(qw.astype(np.uint64), oq.w)
    # both deduplication methods give the same quotient CSR
    for mode in (cd.QUOTIENT_SORT, cd.QUOTIENT_DENSE):
        qm = cd.quotient_build(cd.cluster(g, tau, seed, delta0_mode=mode_d0, quotient_mode=mode))
        moff, mcol, mw = qm.copy()
        assert np.array_equal(moff, qoff) and np.array_equal(mcol, qcol) and np.array_equal(mw, qw), mode
    r = cd.estimate(q)
    ores = oracle.estimate(oq, ocl)
    assert (r["k"], r["phi_gc"], r["radius"], r["phi_approx"]) == (ores.k, ores.phi_gc, ores.radius, ores.phi_approx)
    return r


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("lcc", [True, False])
def test_csr_random(cd, seed, lcc):
    check_csr(cd, *rand_edges(seed), lcc)


@pytest.mark.parametrize("n,wmax", [(200_000, 0xFFFFFFFF), (70_000, 1 << 31), (1 << 16, 0xFFFFFFFF), (5, 0xFFFFFFFF),
                                    (1 << 20, 1 << 24), (1 << 20, (1 << 24) - 1)])
def test_csr_wide_items(cd, n, wmax):
    # 2 * bits(n - 1) + bits(max w) > 64 takes the (key, weight) pair path, <= 64 the packed-word path
    m = 3 * n
    rng = np.random.default_rng(n)
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    w = rng.integers(1, wmax, m, dtype=np.uint64, endpoint=True).astype(np.uint32)
    w[:4] = wmax  # the largest weight is present
    check_csr(cd, n, src, dst, w, False)


@pytest.mark.parametrize("case", ["long_runs", "loops_tail", "sparse_rows", "tile_edges"])
@pytest.mark.parametrize("lcc", [True, False])
def test_csr_dedup_tile_boundaries(cd, case, lcc):
    # de-duplication runs 2048 sorted items per tile: runs of one (row, col) spanning several tiles,
    # dropped self-loops filling whole tiles at the end, rows with no entries, item counts at tile edges
    rng = np.random.default_rng(["long_runs", "loops_tail", "sparse_rows", "tile_edges"].index(case))
    if case == "long_runs":
        n = 300
        src = np.concatenate([np.full(6000, 7), np.full(2100, 8), rng.integers(0, n, 3000)]).astype(np.uint32)
        dst = np.concatenate([np.full(6000, 9), np.full(2100, 7), rng.integers(0, n, 3000)]).astype(np.uint32)
        perm = rng.permutation(src.size)
        src, dst = src[perm], dst[perm]
    elif case == "loops_tail":
        n = 500
        a = rng.integers(0, n, 7000)
        src = np.concatenate([a, rng.integers(0, n, 900)]).astype(np.uint32)
        dst = np.concatenate([a, rng.integers(0, n, 900)]).astype(np.uint32)
    elif case == "sparse_rows":
        n = 200_000
        src = rng.integers(0, n, 5000).astype(np.uint32)
        dst = (src + rng.integers(1, 4, 5000)).astype(np.uint32) % n
    else:
        for m in (1023, 1024, 1025, 2048, 2049):
            n = 64
            src = rng.integers(0, n, m).astype(np.uint32)
            dst = rng.integers(0, n, m).astype(np.uint32)
            w = rng.integers(1, 1000, m).astype(np.uint32)
            check_csr(cd, n, src, dst, w, lcc)
        return
    w = rng.integers(1, 1 << 20, src.size).astype(np.uint32)
    check_csr(cd, n, src, dst, w, lcc)


def test_csr_degenerate(cd):
    z = np.zeros(0, np.uint32)
    g = cd.build_csr(z, z, z, 1)
    assert g.n == 1 and g.nnz == 0
    s = np.array([0, 1, 2], np.uint32)
    g = cd.build_csr(s, s, np.ones(3, np.uint32), 3)
    assert g.n == 1 and g.nnz == 0
    with pytest.raises(cd.CldiamError):
        cd.build_csr(np.array([0], np.uint32), np.array([5], np.uint32), np.array([1], np.uint32), 3)
    with pytest.raises(cd.CldiamError):
        cd.build_csr(np.array([0], np.uint32), np.array([1], np.uint32), np.array([0], np.uint32), 3)


@pytest.mark.parametrize("seed", range(12))
def test_cluster_random_connected(cd, seed):
    n, s, d, w = rand_edges(100 + seed)
    g, og = check_csr(cd, n, s, d, w, True)
    for tau in (0.05, 0.3):
        check_cluster(cd, g, og, tau, seed)
    check_cluster(cd, g, og, 0.1, seed, mode=1)


@pytest.mark.parametrize("seed", range(8))
def test_cluster_disconnected_guard(cd, seed):
    # no LCC: some components start without a center, which exercises the fixed-point guard
    n, s, d, w = rand_edges(200 + seed, n=300, m=200)
    g, og = check_csr(cd, n, s, d, w, False)
    check_cluster(cd, g, og, 0.2, seed)


def test_cluster_all_singletons(cd):
    n, s, d, w = rand_edges(7, n=50, m=120)
    g, og = check_csr(cd, n, s, d, w, True)
    r = check_cluster(cd, g, og, 1e6, 3)
    assert r["k"] == g.n and r["stages"] == 0


def test_single_node(cd):
    z = np.zeros(0, np.uint32)
    g = cd.build_csr(z, z, z, 1)
    c = cd.cluster(g, 1.0, 1)
    r = cd.estimate(cd.quotient_build(c))
    assert r["k"] == 1 and r["phi_approx"] == 0


@pytest.mark.parametrize("side,W", [(16, 10), (33, 100), (64, 100)])
def test_meshes(cd, side, W):
    e = inputs.grid(side, W, side)
    g, og = check_csr(cd, e.n, e.src, e.dst, e.w, True)
    for tau in (0.1, 0.3, 1.0):
        check_cluster(cd, g, og, tau, side)


@pytest.mark.parametrize("scale", [8, 11, 14])
def test_rmat(cd, scale):
    e = inputs.rmat(scale, 8, 1000, scale)
    g, og = check_csr(cd, e.n, e.src, e.dst, e.w, True)
    for tau in (0.5, 2.0):
        check_cluster(cd, g, og, tau, scale)


def test_road_mesh(cd):
    e = inputs.road_mesh(128, 1000, 3)
    g, og = check_csr(cd, e.n, e.src, e.dst, e.w, True)
    check_cluster(cd, g, og, 0.5, 3)


def test_grid64_workload(cd):
    from inputs.workloads import WORKLOADS
    wl = WORKLOADS["grid64"]
    e = wl.make()
    g, og = check_csr(cd, e.n, e.src, e.dst, e.w, True)
    r = check_cluster(cd, g, og, wl.tau, wl.seed)
    assert r["phi_approx"] >= 3164  # >= the farthest-node lower bound of this mesh (oracle, 4 sweeps)


@pytest.mark.parametrize("seed", range(6))
def test_sssp_delta(cd, seed):
    n, s, d, w = rand_edges(300 + seed, wmax=1000)
    g, og = check_csr(cd, n, s, d, w, False)
    src = cd.sssp_source(g, seed)
    assert src == oracle.sssp_source(seed, g.n)
    ref = oracle.dijkstra(og, src)
    for delta in (0, 1, 37, 5000):
        dist, ecc, rounds = cd.sssp_delta(g, src, delta)
        ref32 = np.where(ref == oracle.UNREACHABLE, 0xFFFFFFFF, ref).astype(np.uint64)
        assert np.array_equal(dist.astype(np.uint64), ref32)
        assert ecc == int(ref[ref != oracle.UNREACHABLE].max())


def test_sssp_workload_shapes(cd):
    for e in (inputs.grid(64, 100, 1), inputs.rmat(14, 16, 1 << 20, 2), inputs.road_mesh(96, 1000, 3)):
        g, og = check_csr(cd, e.n, e.src, e.dst, e.w, True)
        src = cd.sssp_source(g, 5)
        dist, ecc, _ = cd.sssp_delta(g, src)
        assert np.array_equal(dist.astype(np.uint64), oracle.dijkstra(og, src))


@pytest.mark.parametrize("seed", range(5))
def test_apsp_max(cd, seed):
    rng = np.random.default_rng(seed)
    for k in (1, 2, 31, 32, 33, 70):
        n, s, d, w = rand_edges(seed * 100 + k, n=k, m=3 * k, wmax=1 << 20)
        og = oracle.build_csr(n, s, d, w, lcc=False)
        q = oracle.Quotient(og.n, np.arange(og.n, dtype=np.uint32), og.off, og.col, og.wt.astype(np.uint64))
        assert cd.apsp_max(og.n, og.off, og.col, og.wt) == oracle.apsp_max(q)


@pytest.mark.parametrize("k", [65, 130, 200])
def test_apsp_dense_floyd_warshall(cd, k):
    # a dense quotient (>= k^2/8 entries) takes the blocked Floyd-Warshall path, across several 64-wide tiles
    rng = np.random.default_rng(k)
    iu = np.triu_indices(k, 1)
    keep = rng.random(iu[0].size) < 0.6
    s, d = iu[0][keep].astype(np.uint32), iu[1][keep].astype(np.uint32)
    w = rng.integers(1, 1 << 20, s.size).astype(np.uint32)
    og = oracle.build_csr(k, s, d, w, lcc=False)
    assert og.nnz * 8 >= k * k
    q = oracle.Quotient(og.n, np.arange(og.n, dtype=np.uint32), og.off, og.col, og.wt.astype(np.uint64))
    assert cd.apsp_max(og.n, og.off, og.col, og.wt) == oracle.apsp_max(q)


def _dense(k, seed, lo, hi, blocks=1):
    # dense random graph on k nodes (>= k^2/8 entries), optionally split into disconnected blocks
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(k, 1)
    keep = rng.random(iu[0].size) < 0.6
    if blocks > 1:
        keep &= (iu[0] * blocks // k) == (iu[1] * blocks // k)
    s, d = iu[0][keep].astype(np.uint32), iu[1][keep].astype(np.uint32)
    w = rng.integers(lo, hi, s.size, dtype=np.uint64, endpoint=True).astype(np.uint32)
    og = oracle.build_csr(k, s, d, w, lcc=False)
    q = oracle.Quotient(og.n, np.arange(og.n, dtype=np.uint32), og.off, og.col, og.wt.astype(np.uint64))
    return og, q


@pytest.mark.parametrize("k,blocks,lo,hi", [
    (150, 2, 1, 1 << 20),                      # disconnected: the fast form leaves pairs unconnected
    (140, 1, 1 << 30, 0x7FFFFFFE),             # distances past 2^31 - 1: the fast form cannot hold them
    (130, 1, 0x7FFFFFFF, 0x7FFFFFFF + 100),    # weights the fast form cannot hold at all
])
def test_apsp_dense_checked_form(cd, k, blocks, lo, hi):
    # the fast Floyd-Warshall form must hand over to the checked form, which is exact or refuses:
    # exact whenever every distance is below 2^31 - 1 or no candidate sum reaches 2^32 - 1; a
    # candidate sum that reaches 2^32 - 1 is reported as OVERFLOW (never a wrapped value)
    og, q = _dense(k, k + blocks, lo, hi, blocks)
    assert og.nnz * 8 >= k * k
    ref = oracle.apsp_max(q)
    try:
        got = cd.apsp_max(og.n, og.off, og.col, og.wt)
    except cd.CldiamError as ex:
        assert ex.status == -3 and ref >= 0x7FFFFFFF, (ex, hex(ref))
        return
    assert got == ref
    if blocks > 1:
        assert ref < 0x7FFFFFFF  # the disconnected case is answered exactly


def test_apsp_dense_overflow_reported(cd):
    # chain-like dense graph whose diameter exceeds 2^32 - 1: OVERFLOW, never a wrapped value
    k = 70
    s = np.arange(k - 1, dtype=np.uint32); d = s + 1
    w = np.full(k - 1, 0x10000000, np.uint32)  # 69 x 2^28 > 2^32
    rng = np.random.default_rng(3)
    iu = np.triu_indices(k, 2)
    keep = rng.random(iu[0].size) < 0.3
    s = np.concatenate([s, iu[0][keep].astype(np.uint32)]); d = np.concatenate([d, iu[1][keep].astype(np.uint32)])
    w = np.concatenate([w, np.full(int(keep.sum()), 0xFFFFFFF0, np.uint32)])
    og = oracle.build_csr(k, s, d, w, lcc=False)
    assert og.nnz * 8 >= k * k
    q = oracle.Quotient(og.n, np.arange(og.n, dtype=np.uint32), og.off, og.col, og.wt.astype(np.uint64))
    ref = oracle.apsp_max(q)
    if ref >= 0xFFFFFFFF:
        with pytest.raises(cd.CldiamError) as ei:
            cd.apsp_max(og.n, og.off, og.col, og.wt)
        assert ei.value.status == -3
    else:
        assert cd.apsp_max(og.n, og.off, og.col, og.wt) == ref


@pytest.mark.parametrize("k,density,seed", [(3000, 0.002, 6), (2500, 0.003, 7), (700, 0.01, 5)])
def test_apsp_sparse_batched_sssp(cd, k, density, seed):
    # sparse graphs (possibly disconnected) take the multi-source Bellman-Ford path; many rounds
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(k, 1)
    keep = rng.random(iu[0].size) < density
    s, d = iu[0][keep].astype(np.uint32), iu[1][keep].astype(np.uint32)
    w = rng.integers(1, 1 << 20, s.size).astype(np.uint32)
    og = oracle.build_csr(k, s, d, w, lcc=False)
    assert og.nnz * 8 < k * k
    q = oracle.Quotient(og.n, np.arange(og.n, dtype=np.uint32), og.off, og.col, og.wt.astype(np.uint64))
    ref = oracle.apsp_max(q)
    for _ in range(3):
        assert cd.apsp_max(og.n, og.off, og.col, og.wt) == ref


def test_apsp_rejects_malformed_csr(cd):
    off = np.array([0, 2, 1, 3], np.uint64)  # decreasing offsets
    with pytest.raises(cd.CldiamError):
        cd.apsp_max(3, off, np.array([1, 2, 0], np.uint32), np.array([1, 1, 1], np.uint32))
    off = np.array([0, 1, 2, 3], np.uint64)
    with pytest.raises(cd.CldiamError):   # column id out of range
        cd.apsp_max(3, off, np.array([1, 7, 0], np.uint32), np.array([1, 1, 1], np.uint32))


def test_overflow_is_reported(cd):
    # a path whose length exceeds 2^32 - 1: the SSSP must refuse, not wrap
    n = 4
    s = np.array([0, 1, 2], np.uint32); d = np.array([1, 2, 3], np.uint32)
    w = np.array([0xF0000000, 0xF0000000, 5], np.uint32)
    g = cd.build_csr(s, d, w, n)
    with pytest.raises(cd.CldiamError) as ei:
        cd.sssp_delta(g, 0)
    assert ei.value.status == -3


def test_determinism(cd):
    e = inputs.rmat(12, 8, 1000, 9)
    g = cd.build_csr(e.src, e.dst, e.w, e.n)
    a = cd.cluster(g, 1.0, 4).copy()
    b = cd.cluster(g, 1.0, 4).copy()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_run_entry_point(cd):
    e = inputs.grid(40, 100, 2)
    r = cd.run(e.src, e.dst, e.w, e.n, 0.3, 2)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    ores, _, _ = oracle.cldiam(og, 0.3, 2)
    assert (r["k"], r["phi_approx"]) == (ores.k, ores.phi_approx)


def test_device_inputs(cd):
    torch = pytest.importorskip("torch")
    e = inputs.grid(32, 100, 3)
    t = [torch.from_numpy(a.astype(np.int32)).cuda() for a in (e.src, e.dst, e.w)]
    g = cd.build_csr(t[0], t[1], t[2], e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    off, col, w, _ = g.copy()
    assert np.array_equal(off, og.off) and np.array_equal(col, og.col)


def test_pinned_host_inputs(cd):
    # pinned host edge arrays are read in place by the emission kernel (no staging copy)
    torch = pytest.importorskip("torch")
    e = inputs.rmat(12, 8, 1000, 6)
    t = [torch.from_numpy(a.view(np.int32).copy()).pin_memory() for a in (e.src, e.dst, e.w)]
    g = cd.build_csr(t[0], t[1], t[2], e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, e.w)
    off, col, w, orig = g.copy()
    assert np.array_equal(off, og.off) and np.array_equal(col, og.col) and np.array_equal(w, og.wt)
    assert np.array_equal(orig, og.orig)
    r = cd.run(t[0], t[1], t[2], e.n, 0.8, 5)
    ores, _, _ = oracle.cldiam(og, 0.8, 5)
    assert (r["k"], r["phi_approx"]) == (ores.k, ores.phi_approx)


def test_initial_delta_experiment_small(cd):
    # Section 5's initial-Delta experiment on a small two-weight mesh: both starts agree with the
    # oracle, and starting at the diameter gives a much worse ratio than starting at the minimum weight
    e = inputs.grid(128, 10, 7)
    w = np.where(e.w == 1, 1_000_000, 1).astype(np.uint32)
    g = cd.build_csr(e.src, e.dst, w, e.n)
    og = oracle.build_csr(e.n, e.src, e.dst, w)
    lb, _ = oracle.lower_bound(og, 0)
    ratios = []
    for mode, d0 in ((cd.DELTA0_MIN, 0), (cd.DELTA0_EXPLICIT, lb)):
        r = cd.estimate(cd.quotient_build(cd.cluster(g, 0.5, 3, delta0_mode=mode, delta0=d0)))
        ocl = oracle.cluster(og, 0.5, 3, oracle.delta0(og, oracle.DELTA0_MIN) if d0 == 0 else d0)
        ores = oracle.estimate(oracle.quotient(og, ocl), ocl)
        assert (r["k"], r["phi_approx"], r["steps"]) == (ores.k, ores.phi_approx, ocl.stats["steps"])
        ratios.append(r["phi_approx"] / lb)
    assert ratios[0] < 1.01 and ratios[1] > 2.0, ratios
