"""Seeded input generators: shapes, determinism, weight law (inputs only)."""
import numpy as np

import inputs


def test_grid_shape_and_weights():
    e = inputs.grid(64, 100, 1)
    assert e.n == 4096 and e.m == 8064
    assert e.w.min() >= 1 and e.w.max() <= 100
    assert np.all(e.src < e.dst)
    e2 = inputs.grid(64, 100, 1)
    assert np.array_equal(e.w, e2.w)
    assert not np.array_equal(e.w, inputs.grid(64, 100, 2).w)


def test_rmat_shape_and_skew():
    e = inputs.rmat(12, 16, 1 << 20, 2)
    assert e.n == 4096 and e.m == 16 * 4096
    assert e.src.max() < e.n and e.dst.max() < e.n
    deg = np.bincount(np.concatenate([e.src, e.dst]), minlength=e.n)
    assert deg.max() > 20 * np.median(deg)          # power-law skew
    assert np.array_equal(e.src, inputs.rmat(12, 16, 1 << 20, 2).src)


def test_road_mesh():
    e = inputs.road_mesh(100, 1000, 3)
    mg = 2 * 100 * 99
    kept = e.m - int(0.001 * mg)
    assert abs(kept / mg - 0.9) < 0.02
    assert e.w.max() <= 1000


def test_mix_and_queries():
    kinds = [inputs.mix_params(4, g)[0] for g in range(400)]
    assert 0.4 < np.mean(kinds) < 0.6
    for g in range(50):
        kind, scale, side, _ = inputs.mix_params(4, g)
        assert 8 <= scale <= 16 and 32 <= side <= 512
    t, gi = inputs.queries(5, 2000, 100.0, 0.01, 2000)
    assert np.all(np.diff(t) > 0) and abs(t[-1] / 2000 - 0.01) < 0.002
    assert 0 < (gi == 2000).sum() < 60
