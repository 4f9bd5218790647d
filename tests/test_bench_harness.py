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


def test_clock_summary_keeps_the_timed_window():
    """The clock record covers the timed region only: samples before and after it (warm-up,
    the next leg) are left out, and their reasons too."""
    import bench
    cs = bench.ClockSampler(0)
    cs.max_mhz = 2070.0
    cs.samples = [(0.90, 1500.0, ["sw_thermal_slowdown"]),  # warm-up, before the region
                  (1.00, 2070.0, []), (1.01, 2055.0, ["sw_power_cap"]), (1.02, 2070.0, []),
                  (1.20, 900.0, ["hw_slowdown"])]  # after the region
    s = cs.summary(0.995, 1.025)
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["window_ms"] == 30.0
    # a region shorter than the sampling period: the nearest sample stands in, samples = 0
    s = cs.summary(1.05, 1.06)
    assert s["samples"] == 0 and s["sm_mhz"] == 2070.0 and s["reasons"] == []
    assert cs.summary()["samples"] == 5


def test_clock_sampler_without_nvml_or_nvidia_smi(monkeypatch):
    """On a host with neither NVML nor nvidia-smi the sampler records nothing and says so."""
    import bench
    monkeypatch.setenv("PATH", "/nonexistent")
    cs = bench.ClockSampler(0)
    monkeypatch.setattr(cs, "_nvml_open", lambda: (_ for _ in ()).throw(OSError("no NVML")))
    with cs:
        pass
    s = cs.summary(0.0, 1.0)
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["source"] is None
