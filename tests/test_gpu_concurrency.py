"""Calls from several host threads on their own streams at once: the library keeps no per-call state
outside its handles (profiling, tuning, pinned blocks and launch attributes are behind locks or atomics),
so concurrent calls give exactly the one-call results.  Inputs: pinned host edge lists (copied to the
device by the copy engine on each call's stream) and device arrays, mixed."""
import threading

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cd():
    import paper_1506_03265_gb300 as m
    m.load()
    m.tuning_set()
    yield m


def run_threads(fn, count):
    outs, errs = [None] * count, []

    def work(j):
        try:
            outs[j] = fn(j)
        except Exception as ex:
            errs.append(ex)

    threads = [threading.Thread(target=work, args=(j,)) for j in range(count)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errs:
        raise errs[0]
    return outs


def test_concurrent_runs_match_one_run(cd):
    import torch
    graphs = [inputs.rmat(14, 16, 1000, 3), inputs.road_mesh(128, 1000, 2)]
    taus = [1.0, 0.5]
    host = [[torch.from_numpy(a.view(np.int32)).pin_memory() for a in (e.src, e.dst, e.w)] for e in graphs]
    dev = [[t.cuda() for t in h] for h in host]
    ref = [cd.run(*host[i], graphs[i].n, taus[i], 5) for i in range(len(graphs))]
    assert ref[0] == cd.run(*dev[0], graphs[0].n, taus[0], 5)  # the host-link and device inputs agree
    streams = [torch.cuda.Stream() for _ in range(4)]

    def job(j):
        i = j % len(graphs)
        arrays = host[i] if j < 2 else dev[i]
        return [cd.run(*arrays, graphs[i].n, taus[i], 5, stream=streams[j]) for _ in range(3)]

    outs = run_threads(job, 4)
    torch.cuda.synchronize()
    for j, rs in enumerate(outs):
        assert all(r == ref[j % len(graphs)] for r in rs), j


def test_concurrent_handles_on_their_own_streams(cd):
    import torch
    e = inputs.rmat(13, 8, 1000, 7)
    g_ref = cd.build_csr(e.src, e.dst, e.w, e.n)
    c_ref = cd.cluster(g_ref, 0.8, 2)
    ref_cl = c_ref.copy()
    ref_est = cd.estimate(cd.quotient_build(c_ref))
    streams = [torch.cuda.Stream() for _ in range(3)]

    def job(j):
        g = cd.build_csr(e.src, e.dst, e.w, e.n, stream=streams[j])
        c = cd.cluster(g, 0.8, 2)
        return c.copy(), cd.estimate(cd.quotient_build(c))

    for cl, est in run_threads(job, 3):
        assert all(np.array_equal(a, b) for a, b in zip(cl, ref_cl)) and est == ref_est
