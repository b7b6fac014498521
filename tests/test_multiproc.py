"""Replica (weak-scaling) path of bench.py on two gloo ranks on CPU: problems
are sharded without any data-path collective, and the step time is the
maximum over ranks."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        items = list(range(11))
        mine = bench.shard(items, ws, rank)
        t = bench.max_over_ranks(1.5 + rank, ws)
        q.put((rank, mine, t))
    finally:
        dist.destroy_process_group()


def test_replica_sharding_and_max_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = 2
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(11))
    assert not set(shards[0]) & set(shards[1])
    assert all(r[2] == 2.5 for r in res)


def test_single_rank_helpers():
    import bench
    assert bench.shard([1, 2, 3], 1, 0) == [1, 2, 3]
    assert bench.max_over_ranks(3.0, 1) == 3.0
