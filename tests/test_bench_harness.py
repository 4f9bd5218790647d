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


def test_committed_trace_profile_matches_the_kernel_sources():
    """The roofline's DRAM traffic and the issue roof's instructions per ray come from the
    committed ncu summary of the BVH2 trace kernel; the summary names the sources it was
    captured from by hash, and a changed kernel or tree builder must be recaptured."""
    import bench
    assert bench.profile_traffic() is not None, "trace kernel sources changed since profiles/ was captured"
    assert 300 < bench.profile_traffic("warp_instructions_per_ray") < 500


def test_roofline_arithmetic():
    """Bytes per ray and the issue roof, recomputed by hand from the figures of a bench line
    (40.17 BVH2 nodes and 4.32 triangles per secondary ray; 152 SMs at 2070 MHz)."""
    import bench
    assert abs(bench.trace_bytes_per_ray(40.17, 4.32) - (44 + 64 * 40.17 + 48 * 4.32)) < 1e-9
    assert abs(bench.trace_bytes_per_ray(40.17, 4.32) - 2822.24) < 1e-6
    assert bench.trace_bytes_per_ray(21.0, 4.4, 112) == 44 + 112 * 21.0 + 48 * 4.4
    r = bench.issue_roof({"trace_mrays": 1850.0}, 2070.0, 152)
    assert abs(r["peak"] - 152 * 4 * 2070e6 / 1e12) < 1e-3
    ipr = bench.profile_traffic("warp_instructions_per_ray")
    assert abs(r["achieved"] - round(ipr * 1850e6 / 1e12, 3)) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
