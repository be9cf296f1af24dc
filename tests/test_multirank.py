"""Multi-process host logic of the many-graph form, with world_size-2 gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1506_03265_gb300.shard import lpt_partition, max_over_ranks, sum_over_ranks  # noqa: E402


def test_lpt_partition_covers_and_balances():
    w = [5, 1, 1, 1, 9, 2, 2, 7, 3, 3]
    parts = lpt_partition(w, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w)))
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)
    assert lpt_partition(w, 1) == [list(range(len(w)))]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        weights = [float((i * 37) % 11 + 1) for i in range(50)]
        parts = lpt_partition(weights, world)          # computed independently on every rank
        mine = parts[rank]
        local_time = 1.0 + rank                          # rank 1 is the slowest
        tmax = max_over_ranks(local_time, dist)
        total = sum_over_ranks(len(mine), dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, tmax, total, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, total, gathered in out:
        assert tmax == 2.0 and total == 50
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(50))                  # every graph on exactly one rank
    assert out[0][3] == out[1][3]                        # identical partitions on both ranks
