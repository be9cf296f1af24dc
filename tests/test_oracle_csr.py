"""Pin the oracle's CSR builder (graph model of Section 2) against numpy/scipy.

Independent restatement: dedup unordered pairs keeping the minimum weight with
numpy lexsort/unique, drop self-loops, mirror, sort; LCC with scipy's
connected_components.
"""
import numpy as np
import pytest

import inputs
import oracle

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def ref_csr(n, src, dst, w, lcc):
    src = src.astype(np.int64); dst = dst.astype(np.int64); w = w.astype(np.int64)
    keep = src != dst
    a = np.minimum(src, dst)[keep]; b = np.maximum(src, dst)[keep]; ww = w[keep]
    order = np.lexsort((ww, b, a))
    a, b, ww = a[order], b[order], ww[order]
    if a.size:
        first = np.ones(a.size, bool)
        first[1:] = (a[1:] != a[:-1]) | (b[1:] != b[:-1])
        a, b, ww = a[first], b[first], ww[first]
    r = np.concatenate([a, b]); c = np.concatenate([b, a]); x = np.concatenate([ww, ww])
    o = np.lexsort((c, r))
    r, c, x = r[o], c[o], x[o]
    keep_nodes = np.arange(n)
    if lcc:
        M = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(n, n)).tocsr()
        ncomp, lab = csgraph.connected_components(M, directed=False)
        sizes = np.bincount(lab, minlength=ncomp)
        # largest; ties -> component containing the smallest node id
        best = max(range(ncomp), key=lambda L: (sizes[L], -np.flatnonzero(lab == L)[0]))
        keep_nodes = np.flatnonzero(lab == best)
        newid = -np.ones(n, np.int64); newid[keep_nodes] = np.arange(keep_nodes.size)
        sel = newid[r] >= 0
        r, c, x = newid[r[sel]], newid[c[sel]], x[sel]
    nk = keep_nodes.size
    off = np.zeros(nk + 1, np.uint64)
    np.add.at(off, r + 1, 1)
    off = np.cumsum(off).astype(np.uint64)
    return nk, off, c.astype(np.uint32), x.astype(np.uint32), keep_nodes.astype(np.uint32)


def check(n, src, dst, w, lcc):
    g = oracle.build_csr(n, src, dst, w, lcc=lcc)
    nk, off, col, wt, orig = ref_csr(n, src, dst, w, lcc)
    assert g.n == nk
    assert np.array_equal(g.off, off)
    assert np.array_equal(g.col, col)
    assert np.array_equal(g.wt, wt)
    assert np.array_equal(g.orig, orig)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("lcc", [False, True])
def test_random_multigraphs(seed, lcc):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    m = int(rng.integers(0, 200))
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    w = rng.integers(1, 5, m).astype(np.uint32)   # small range forces duplicate pairs with distinct weights
    check(n, src, dst, w, lcc)


def test_generators_through_builder():
    for e in [inputs.grid(9, 100, 1), inputs.rmat(8, 8, 1000, 3), inputs.road_mesh(12, 1000, 3)]:
        check(e.n, e.src, e.dst, e.w, True)


def test_degenerate():
    z = np.zeros(0, np.uint32)
    g = oracle.build_csr(1, z, z, z, lcc=True)
    assert g.n == 1 and g.nnz == 0
    # only self-loops: every node is its own component; the LCC is node 0
    s = np.array([0, 1, 2], np.uint32)
    g = oracle.build_csr(3, s, s, np.ones(3, np.uint32), lcc=True)
    assert g.n == 1 and g.nnz == 0 and g.orig[0] == 0
    # two equal components: the one holding the smallest id wins
    g = oracle.build_csr(4, np.array([2, 0], np.uint32), np.array([3, 1], np.uint32),
                         np.array([5, 7], np.uint32), lcc=True)
    assert list(g.orig) == [0, 1] and list(g.wt) == [7, 7]


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.build_csr(2, np.array([0], np.uint32), np.array([1], np.uint32), np.array([0], np.uint32))
    with pytest.raises(ValueError):
        oracle.build_csr(2, np.array([0], np.uint32), np.array([2], np.uint32), np.array([1], np.uint32))


def test_delta0():
    e = inputs.grid(10, 100, 4)
    g = oracle.build_csr(e.n, e.src, e.dst, e.w)
    upper = g.col > np.repeat(np.arange(g.n), np.diff(g.off).astype(np.int64))
    assert oracle.delta0(g, oracle.DELTA0_AVG) == max(1, int(g.wt[upper].astype(np.int64).sum()) // int(upper.sum()))
    assert oracle.delta0(g, oracle.DELTA0_MIN) == int(g.wt.min())
