"""Host-side logic of the multi-rank benchmark on CPU: two gloo ranks render disjoint frames
and the timing aggregates are max (time) and sum (rays) over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    import bench
    frames = [bench.frame_of(rank, s, world) for s in range(5)]
    t_max = bench.aggregate(1.5 + rank, "max")
    rays = bench.aggregate(100.0 * (rank + 1), "sum")
    bench.barrier()
    q.put((rank, frames, t_max, rays, bench.dist_info()))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f0, f1 = res[0][1], res[1][1]
    assert not set(f0) & set(f1)  # ranks render disjoint frames
    assert sorted(f0 + f1) == list(range(10))
    for r in res:
        assert r[2] == 2.5 and r[3] == 300.0
    assert res[1][4] == (1, 2, 1)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate(3.25, "max") == 3.25
    assert bench.frame_of(0, 7, 1) == 7
