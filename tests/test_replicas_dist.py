"""The multi-GPU mode is replicas only (independent lattices per rank, no
data-path collective).  Its host logic -- disjoint replica seeds per rank and
the max-over-ranks timing reduction -- runs here with world size 2 over gloo
on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + rank, 20.0 - rank]
    got = bench.max_over_ranks(local, dist, "cpu")
    q.put((rank, bench.replica_seed(rank, 4), got))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_seeds_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][2] == res[1][2] == [11.0, 20.0]
    assert res[0][1] != res[1][1] and abs(res[0][1] - res[1][1]) == 4
