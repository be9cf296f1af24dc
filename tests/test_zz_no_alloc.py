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


def test_rejects_what_it_cannot_serve(env):
    torch, cd = env
    off, col, w = symmetric_csr(1100, 0.5, 7)     # dense and above the 1024 limit
    d = [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda() for a in (off, col, w)]
    with pytest.raises(cd.CldiamError) as ei:
        cd.apsp_max_noalloc(1100, d[0], d[1], d[2])
    assert ei.value.status == -9
    off, col, w = symmetric_csr(50, 0.5, 8)       # host arrays: nothing is copied, so they are refused
    with pytest.raises(cd.CldiamError) as ei:
        cd.apsp_max_noalloc(50, off, col, w)
    assert ei.value.status == -1
