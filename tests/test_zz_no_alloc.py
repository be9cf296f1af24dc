"""The allocation-free quotient-diameter entry point (cldiam_apsp_max_noalloc).

Some callers may not allocate GPU memory at all (an application that owns the
device memory budget through its own allocator, or a path that must not risk
an allocation failure mid-run).  This entry point serves them with a fixed
scratch array inside the library.  Each case is checked against the ordinary
cldiam_apsp_max, bit-exactly (the results are integers), on two calls in a
row, since the shared scratch keeps the previous call's contents.  Collected
last so a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def symmetric_csr(k, density, seed, wmax=1 << 20):
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(k, 1)
    keep = rng.random(iu[0].size) < density
    a, b = iu[0][keep], iu[1][keep]
    w = rng.integers(1, wmax, a.size)
    rows = np.concatenate([a, b]); cols = np.concatenate([b, a]); ws = np.concatenate([w, w])
    o = np.lexsort((cols, rows))
    rows, cols, ws = rows[o], cols[o], ws[o]
    off = np.zeros(k + 1, np.uint64)
    np.add.at(off, rows + 1, 1)
    return np.cumsum(off).astype(np.uint64), cols.astype(np.uint32), ws.astype(np.uint32)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import paper_1506_03265_gb300 as cd
    cd.load()
    return torch, cd


# dense graphs take the Floyd-Warshall path in the fixed scratch matrix, sparse ones the
# shared-memory batched SSSP; sizes span one to several 64-wide tiles and a ragged tail
CASES = [(2, 1.0, 1), (64, 0.5, 2), (200, 0.6, 3), (1000, 0.3, 4), (700, 0.01, 5), (3000, 0.002, 6)]


@pytest.mark.parametrize("k,density,seed", CASES)
def test_matches_allocating_entry_point_twice(env, k, density, seed):
    torch, cd = env
    off, col, w = symmetric_csr(k, density, seed)
    d = [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda() for a in (off, col, w)]
    stream = torch.cuda.current_stream()
    ref = cd.apsp_max(k, off, col, w)
    for _ in range(2):
        got = cd.apsp_max_noalloc(k, d[0], d[1], d[2], stream=stream)
        assert got == ref


def test_alternating_sizes_reuse_scratch(env):
    torch, cd = env
    graphs = [symmetric_csr(300, 0.5, 11), symmetric_csr(90, 0.9, 12), symmetric_csr(300, 0.5, 11)]
    for off, col, w in graphs:
        d = [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda()
             for a in (off, col, w)]
        assert cd.apsp_max_noalloc(off.size - 1, d[0], d[1], d[2]) == cd.apsp_max(off.size - 1, off, col, w)


def clustered_csr(k, comps, size, seed, wmax=1 << 20):
    """k nodes: `comps` random components of `size` nodes scattered over the ids (avg degree ~4), the
    rest isolated.  Sparse, so the shared-memory SSSP paths run at large k with little work."""
    rng = np.random.default_rng(seed)
    ids = rng.permutation(k)[:comps * size].reshape(comps, size)
    a, b = [], []
    for c in ids:
        a.append(c[:-1]); b.append(c[1:])                       # a path keeps each component connected
        x = rng.integers(0, size, 2 * size); y = rng.integers(0, size, 2 * size)
        keep = x != y
        a.append(c[x[keep]]); b.append(c[y[keep]])
    a = np.concatenate(a); b = np.concatenate(b)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pairs = np.unique(lo.astype(np.int64) * k + hi)
    lo, hi = pairs // k, pairs % k
    w = rng.integers(1, wmax, lo.size)
    rows = np.concatenate([lo, hi]); cols = np.concatenate([hi, lo]); ws = np.concatenate([w, w])
    o = np.lexsort((cols, rows))
    rows, cols, ws = rows[o], cols[o], ws[o]
    off = np.zeros(k + 1, np.uint64)
    np.add.at(off, rows + 1, 1)
    return np.cumsum(off).astype(np.uint64), cols.astype(np.uint32), ws.astype(np.uint32)


def to_dev(torch, arrs):
    return [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda() for a in arrs]


# the upper ranges of the sparse path: worklist SSSP with one source per CTA (k = 10,000), then
# all-node rounds with the distances alone in shared memory (k = 20,000 and 40,000; the limit is 51,200)
@pytest.mark.parametrize("k,comps,size,seed", [(10_000, 40, 60, 21), (20_000, 30, 50, 22), (40_000, 20, 40, 23)])
def test_sparse_upper_ranges(env, k, comps, size, seed):
    torch, cd = env
    off, col, w = clustered_csr(k, comps, size, seed)
    d = to_dev(torch, (off, col, w))
    ref = cd.apsp_max(k, off, col, w)
    assert ref > 0
    for _ in range(2):
        assert cd.apsp_max_noalloc(k, d[0], d[1], d[2]) == ref


def test_matches_oracle(env):
    import oracle
    torch, cd = env
    k = 3000
    off, col, w = symmetric_csr(k, 0.002, 6)
    d = to_dev(torch, (off, col, w))
    q = oracle.Quotient(k, np.arange(k, dtype=np.uint32), off, col, w.astype(np.uint64))
    assert cd.apsp_max_noalloc(k, d[0], d[1], d[2]) == oracle.apsp_max(q)


def test_overflow_from_both_entry_points(env):
    # a dense graph whose diameter exceeds 2^32 - 1 (a chain of 2^28 weights plus heavy chords): both entry
    # points report OVERFLOW (status -3) instead of a wrapped value
    torch, cd = env
    k = 70
    s = np.arange(k - 1, dtype=np.int64); t = s + 1
    w = np.full(k - 1, 0x10000000, np.int64)
    rng = np.random.default_rng(3)
    iu = np.triu_indices(k, 2)
    keep = rng.random(iu[0].size) < 0.3
    s = np.concatenate([s, iu[0][keep]]); t = np.concatenate([t, iu[1][keep]])
    w = np.concatenate([w, np.full(int(keep.sum()), 0xFFFFFFF0, np.int64)])
    rows = np.concatenate([s, t]); cols = np.concatenate([t, s]); ws = np.concatenate([w, w])
    o = np.lexsort((cols, rows))
    rows, cols, ws = rows[o], cols[o], ws[o]
    off = np.zeros(k + 1, np.uint64)
    np.add.at(off, rows + 1, 1)
    off = np.cumsum(off).astype(np.uint64); col = cols.astype(np.uint32); wu = ws.astype(np.uint32)
    assert int(off[-1]) * 8 >= k * k  # dense: the Floyd-Warshall path of both
    d = to_dev(torch, (off, col, wu))
    with pytest.raises(cd.CldiamError) as e1:
        cd.apsp_max(k, off, col, wu)
    with pytest.raises(cd.CldiamError) as e2:
        cd.apsp_max_noalloc(k, d[0], d[1], d[2])
    assert e1.value.status == -3 and e2.value.status == -3


def test_rejects_what_it_cannot_serve(env):
    torch, cd = env
    off, col, w = symmetric_csr(1100, 0.5, 7)     # dense and above the 1024 limit
    d = [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda() for a in (off, col, w)]
    with pytest.raises(cd.CldiamError) as ei:
        cd.apsp_max_noalloc(1100, d[0], d[1], d[2])
    assert ei.value.status == -9
    k = 51_201                                    # sparse and above the 51,200 limit
    off, col, w = clustered_csr(k, 4, 20, 9)
    d = to_dev(torch, (off, col, w))
    with pytest.raises(cd.CldiamError) as ei:
        cd.apsp_max_noalloc(k, d[0], d[1], d[2])
    assert ei.value.status == -9
    off, col, w = symmetric_csr(50, 0.5, 8)       # host arrays: nothing is copied, so they are refused
    with pytest.raises(cd.CldiamError) as ei:
        cd.apsp_max_noalloc(50, off, col, w)
    assert ei.value.status == -1
