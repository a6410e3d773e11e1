"""Host logic of the multi-rank benchmark on CPU with gloo, world size 2:
systems are sharded with no overlap and full cover, and the only collective
(outside the timed region) gives the max time and the summed units."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    mine = bench.shard(list(range(11)), rank, ws)
    t, u = bench.reduce_time_units(1.5 + rank, len(mine))
    q.put((rank, mine, t, u))
    dist.destroy_process_group()


def test_shard_and_reduce_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(11))
    assert not set(shards[0]) & set(shards[1])
    for rank, mine, t, u in out:
        assert t == 2.5 and u == 11.0


def test_single_rank_identity():
    import bench
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert bench.reduce_time_units(3.0, 7) == (3.0, 7.0)
