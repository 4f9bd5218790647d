#!/usr/bin/env python
"""Benchmark of the direction-reuse path tracer on the landscape workload.

One step = one full render through the C ABI of the 1920x1080 fBm landscape (2,093,058
triangles, 1 spp, 2 bounces, 8x8 tiles, K = 8, LCG-interleaved groups, FP32 BVH2): ray
generation, primary trace, then per bounce shade + classify + reuse + spawn, group
compaction and the secondary trace, then accumulation and output.  The headline value is
secondary Mrays/s of direction reuse over the whole step (device CUDA events on the render
stream); independent sampling and Morton-sorted reordering are measured the same way and
reported beside it.  Inputs (scene, path state) are resident in HBM before timing and the
L2 is flushed between steps.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under torchrun each
rank renders its own frames of the same workload (weak scaling, no data-path collective).
``--impl reference`` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "secondary Mrays/s"
WORKLOAD = ("landscape 1920x1080, fBm terrain 1024^2 grid (2,093,058 tris), 60/30/10 Lambert/GGX/mirror, "
            "sky env, 1 spp, 2 bounces, 8x8 tiles, K=8, LCG interleave, FP32 BVH2")
TILE, K, SPP, BOUNCES = (8, 8), 8, 1, 2


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def frame_of(rank: int, step: int, world: int) -> int:
    """Frame index rendered by ``rank`` at ``step``: ranks render disjoint frames."""
    return step * world + rank


def aggregate(values, op="max"):
    """Reduce a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(values)
    backend = dist.get_backend()
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(values)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled while the timed region runs.

    NVML is polled directly (the same read-only queries nvidia-smi makes) every ``period_s``
    from a host thread, each sample stamped with ``time.perf_counter()``; ``summary(t0, t1)``
    keeps the samples taken inside the timed region.  A timed region of a few tens of
    milliseconds thus still gets a handful of samples, where nvidia-smi's 100 ms loop sees at
    most one.  Without NVML the sampler falls back to an ``nvidia-smi -lms`` process, whose
    lines are stamped on arrival."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of the NVML API (nvmlClocksEventReason*)
    REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                   0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int, uuid: str | None = None, period_s: float = 0.002):
        self.idx = gpu_index
        self.uuid = uuid
        self.period = period_s
        self.samples = []  # (perf_counter, sm_mhz, reason names)
        self.max_mhz = None
        self.source = None
        self._stop = threading.Event()
        self._thread = None
        self.proc = None

    # ---- NVML ----
    def _nvml_open(self):
        import ctypes
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        rc = 1
        if self.uuid:
            rc = nv.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(self.uuid.encode()), ctypes.byref(h))
        if rc != 0:
            rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(h))
        if rc != 0:
            nv.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:  # 1 = NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        return nv, h, reasons

    def _nvml_loop(self, nv, h, reasons):
        import ctypes
        clk, mask = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.perf_counter()
            if nv.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(clk)) == 0:
                names = []
                if reasons(h, ctypes.byref(mask)) == 0:
                    names = [n for bit, n in self.REASON_BITS.items() if mask.value & bit]
                self.samples.append((t, float(clk.value), names))
            self._stop.wait(self.period)
        nv.nvmlShutdown()

    # ---- nvidia-smi fallback ----
    def _smi_loop(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm, self.max_mhz = float(f[1]), float(f[2])
            except ValueError:
                continue
            self.samples.append((time.perf_counter(), sm,
                                 [n for n, v in zip(names, f[5:9]) if v.lower().startswith("active")]))

    def __enter__(self):
        try:
            nv, h, reasons = self._nvml_open()
            self.source = f"NVML every {self.period * 1e3:g} ms"
            self._thread = threading.Thread(target=self._nvml_loop, args=(nv, h, reasons), daemon=True)
        except (OSError, AttributeError):
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "100"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                return self
            self.source = "nvidia-smi -lms 100"
            self._thread = threading.Thread(target=self._smi_loop, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self._thread:
            self._thread.join(timeout=5)

    def summary(self, t0: float | None = None, t1: float | None = None):
        """Median SM clock and the union of reasons over the samples taken in [t0, t1] (all
        samples when no window is given).  If none fell inside, the sample nearest to the
        window stands in and ``samples`` says 0."""
        inside = [x for x in self.samples if (t0 is None or x[0] >= t0) and (t1 is None or x[0] <= t1)]
        use = inside
        if not inside and self.samples and t0 is not None:
            mid = 0.5 * (t0 + (t1 if t1 is not None else t0))
            use = [min(self.samples, key=lambda x: abs(x[0] - mid))]
        reasons = sorted({n for x in use for n in x[2]})
        out = {"sm_mhz": statistics.median(x[1] for x in use) if use else None, "sm_max_mhz": self.max_mhz,
               "reasons": reasons, "samples": len(inside), "source": self.source}
        if t0 is not None and t1 is not None:
            out["window_ms"] = round((t1 - t0) * 1e3, 1)
        return out


def gpu_uuid(index: int) -> str | None:
    """NVML's name ("GPU-<uuid>") of torch's device ``index``, which need not be NVML's index."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(index).uuid)
    except (AttributeError, RuntimeError):
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source_sha(files=("trace.cu", "trace_common.cuh", "bvh_build.cpp")) -> str:
    """sha256 (16 hex digits) of the sources that define the BVH2 trace kernel and the tree
    it traverses (a new tree changes its traffic and instruction counts)."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2310_07182_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(key="dram_bytes_per_launch_full"):
    """A figure of the trace kernel's committed ncu summary (DRAM bytes per launch by
    default), or None if the kernel source changed since that capture."""
    summ = os.path.join(ROOT, "profiles", "k_trace_bvh2.landscape.txt")
    if not os.path.exists(summ):
        return None
    kv = {}
    with open(summ) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_sha") != kernel_source_sha() or key not in kv:
        return None
    return float(kv[key])


# ---------------------------------------------------------------------------------------
def cpu_oracle_rate(sc, target_s: float, max_tiles=None, mode="direction_reuse", frame_base=0, bounces=None):
    """Time the CPU oracle (all host cores) on a bounded sample of the workload's tiles.
    Returns (secondary Mrays/s, threads, sample description, seconds)."""
    B = BOUNCES if bounces is None else bounces
    import oracle
    O = oracle.Scene(sc)
    cam = sc.camera
    ntx = math.ceil(cam.width / TILE[0])
    nty = math.ceil(cam.height / TILE[1])
    ntiles = ntx * nty
    threads = os.cpu_count() or 1
    # probe, then size the sample for ~target_s
    n = min(ntiles, 8 * threads)
    t0 = time.perf_counter()
    r = oracle.render(O, cam, spp=SPP, max_bounces=B, mode=mode, tile=TILE, k=K, seed=0,
                      frame_base=frame_base, tiles=(0, n), threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(ntiles, max(n, n * target_s / max(dt, 1e-3))))
    if max_tiles:
        n2 = min(n2, max_tiles)
    start = (ntiles - n2) // 2  # a band through the middle of the image
    t0 = time.perf_counter()
    r = oracle.render(O, cam, spp=SPP, max_bounces=B, mode=mode, tile=TILE, k=K, seed=0,
                      frame_base=frame_base, tiles=(start, start + n2), threads=threads)
    dt = time.perf_counter() - t0
    sec = int(r["counters"][1])
    sample = f"{n2} of {ntiles} 8x8 tiles ({100.0 * n2 / ntiles:.1f}% of the image), {mode}, 1 spp, {B} bounces"
    return sec / dt / 1e6, r["threads"], sample, dt


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the host cores."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2310_07182_gb300 import scenes
    sc = scenes.landscape()
    per_step = []
    rays = []
    import oracle
    O = oracle.Scene(sc)
    cam = sc.camera
    ntiles = math.ceil(cam.width / TILE[0]) * math.ceil(cam.height / TILE[1])
    threads = os.cpu_count() or 1
    n = min(ntiles, 600 * threads)  # about 1-3 s of oracle work per step on the host cores
    for s in range(args.warmup + args.steps):
        start = (s * 7919 * n) % (ntiles - n)
        t0 = time.perf_counter()
        r = oracle.render(O, cam, spp=SPP, max_bounces=BOUNCES, mode="direction_reuse", tile=TILE, k=K, seed=0,
                          tiles=(start, start + n), threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per_step.append(dt)
            rays.append(int(r["counters"][1]))
    total_t = sum(per_step)
    value = sum(rays) / total_t / 1e6
    sample = f"{n} of {ntiles} 8x8 tiles per step, direction_reuse, 1 spp, 2 bounces"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * total_t / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": round(value, 4), "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2310_07182_gb300 import binding as cr
    from paper_2310_07182_gb300 import build as crbuild
    from paper_2310_07182_gb300 import scenes
    crbuild.build()
    t_setup = time.perf_counter()
    # --scene interior: the indoor workload with its ceiling light (profiling shadow rays);
    # the headline metric is the landscape's
    sc = scenes.landscape() if args.scene == "landscape" else scenes.interior()
    workload = WORKLOAD if args.scene == "landscape" else "interior 1280x720 (512,014 tris), 1 spp, B=2, 8x8 K=8"
    # a "+bvh8q" ("+bvh4") mode traces through the 8-wide quantised (4-wide FP32) BVH
    S = cr.Scene(sc, bvh_flags=cr.CR_BVH2 | (cr.CR_BVH8Q if "+bvh8q" in args.modes else 0) |
                 (cr.CR_BVH4 if "+bvh4" in args.modes else 0))
    cam = sc.camera
    out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream().cuda_stream
    setup_s = time.perf_counter() - t_setup

    variant_flags = {"two_phase": cr.CR_OPT_TWO_PHASE, "packet": cr.CR_OPT_PACKET_SECONDARY,
                     "speculative": cr.CR_OPT_SPECULATIVE, "persistent": cr.CR_OPT_PERSISTENT,
                     "nee": cr.CR_OPT_NEE, "ordered": cr.CR_OPT_ORDERED_QUEUES}

    def parse(mode):
        # "morton_sort:<key>" selects a reordering key (Table 1 comparators); a "+<variant>"
        # suffix selects a traversal variant of the secondary trace, "+bvh8q" the BVH8-Q and
        # "+bvh4" the BVH4 for every closest-hit trace
        mode, *variants = mode.split("+")
        m, _, key = mode.partition(":")
        flags, bvh = 0, cr.CR_BVH2
        for v in variants:
            if v == "bvh8q":
                bvh = cr.CR_BVH8Q
            elif v == "bvh4":
                bvh = cr.CR_BVH4
            else:
                flags |= variant_flags[v]
        return m, key or "two_point", flags, bvh

    def step(mode, frame, flags=0, stats_flag=None):
        # timed steps record events only around the trace launches (the whole-step time, the
        # trace-only rate and the roofline's launch time); the full per-stage breakdown comes
        # from separate untimed steps, because ~30 event records per step cost ~3% of it
        m, key, vflags, bvh = parse(mode)
        flags |= vflags
        st = cr.cr_stats()
        o = cr.make_opts(k=K, interleave=True, seed=0, frame_base=frame, bvh=bvh,
                         flags=(cr.CR_OPT_STATS_TRACES if stats_flag is None else stats_flag) | flags, stream=stream,
                         stats=st, sort_key=key)
        cr.cr_render_ex(S.handle, cam, SPP, BOUNCES, m, TILE[0], TILE[1], out, o)
        return st.as_dict()

    # counting pass (untimed): node visits and triangle tests of the secondary traces
    modes = args.modes.split(",")
    if not args.core_only and "morton_sort" in modes:  # the other reordering keys of Table 1
        modes += ["morton_sort:origin", "morton_sort:reis", "morton_sort:costa", "morton_sort:aila_compact",
                  "morton_sort:hierarchy_cut"]
    counts = {}
    for mode in modes:
        counts[mode] = step(mode, frame_of(rank, 0, world), flags=cr.CR_OPT_COUNT)

    results = {}
    clocks = None
    sampler = None
    for mode in modes:
        if mode == modes[0]:  # sampling starts before the warm-up so it is live when timing starts
            sampler = ClockSampler(local, uuid=gpu_uuid(local)).__enter__()
        for w in range(args.warmup):  # warm-up steps as the timed ones, L2 flush included
            flush.fill_(float(w))
            step(mode, frame_of(rank, w, world))
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        stats = []
        t_wall = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(float(s))  # evict the L2 between steps (outside the timed events)
            stats.append(step(mode, frame_of(rank, args.warmup + s, world)))
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_end = time.perf_counter()
        wall = t_end - t_wall
        if sampler and mode == modes[0]:
            sampler.__exit__()
            clocks = sampler.summary(t_wall, t_end)
        ms = sum(x["ms_total"] for x in stats)
        ms_max = aggregate(ms, "max")
        sec = sum(x["secondary_rays"] for x in stats)
        sec_all = aggregate(sec, "sum")
        results[mode] = dict(
            mrays=sec_all / (ms_max / 1e3) / 1e6,
            ms_per_step=ms_max / args.steps,
            trace_mrays=sec / (sum(x["ms_trace_secondary"] for x in stats) / 1e3) / 1e6,
            ms_trace_secondary=sum(x["ms_trace_secondary"] for x in stats) / args.steps,
            ms_trace_primary=sum(x["ms_trace_primary"] for x in stats) / args.steps,
            secondary_rays_per_step=sec / args.steps,
            launches_per_step=stats[0]["kernel_launches"],
            wall_s=wall,
        )
        c = counts[mode]
        results[mode]["nodes_per_ray"] = c["node_visits"] / max(c["secondary_rays"], 1)
        results[mode]["tris_per_ray"] = c["tri_tests"] / max(c["secondary_rays"], 1)
        # stage breakdown (untimed steps with events between all stages)
        br = [step(mode, frame_of(rank, args.warmup + args.steps + i, world), stats_flag=cr.CR_OPT_STATS)
              for i in range(3)]
        for key in ("ms_shade", "ms_compact", "ms_sort", "ms_raygen", "ms_accum"):
            results[mode][key] = sum(x[key] for x in br) / len(br)

    # End to end through the C ABI, every step's image read back to page-locked host memory.
    # (1) synchronous: cr_render_ex into the host buffer (staging copy inside the call), one
    # call after the other.  (2) pipelined: double-buffered device images, each copied to its
    # own host buffer on a side stream while the next step renders (how a frame loop
    # overlaps readback with work); all copies finish inside the timed region.
    m0, key0, flags0, bvh0 = parse(modes[0])
    hosts = [torch.empty((cam.height, cam.width, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    devs = [torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    st_io = cr.cr_stats()
    cr.cr_render_ex(S.handle, cam, SPP, BOUNCES, m0, TILE[0], TILE[1], hosts[0],
                    cr.make_opts(k=K, frame_base=frame_of(rank, 0, world), flags=flags0 | cr.CR_OPT_STATS_TRACES,
                                 sort_key=key0, stats=st_io, bvh=bvh0))
    h2d_step = int(st_io.h2d_bytes)

    def e2e_sync(n, s0):
        for s in range(n):
            cr.cr_render_ex(S.handle, cam, SPP, BOUNCES, m0, TILE[0], TILE[1], hosts[0],
                            cr.make_opts(k=K, frame_base=frame_of(rank, s0 + s, world), flags=flags0,
                                         sort_key=key0, bvh=bvh0))

    main_stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_pipelined(n, s0):
        for s in range(n):
            b = s % 2
            main_stream.wait_event(copied[b])  # the copy of step s - 2 has left this buffer
            cr.cr_render_ex(S.handle, cam, SPP, BOUNCES, m0, TILE[0], TILE[1], devs[b],
                            cr.make_opts(k=K, frame_base=frame_of(rank, s0 + s, world),
                                         flags=flags0 | cr.CR_OPT_NO_SYNC, sort_key=key0, bvh=bvh0,
                                         stream=main_stream.cuda_stream))
            rendered[b].record(main_stream)
            copy_stream.wait_event(rendered[b])
            with torch.cuda.stream(copy_stream):
                hosts[b].copy_(devs[b], non_blocking=True)
            copied[b].record(copy_stream)
        copy_stream.synchronize()
        main_stream.synchronize()

    e2e_rays = aggregate(results[modes[0]]["secondary_rays_per_step"] * args.steps, "sum")
    e2e = {}
    for name, fn in (("sync", e2e_sync), ("pipelined", e2e_pipelined)):
        fn(args.warmup, 0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        fn(args.steps, args.warmup)
        e2e[name] = aggregate(time.perf_counter() - t0, "max")

    extras = {}
    # the legs beyond the headline (precision, sweeps, quality, batching, serving) run at
    # N = 1; a multi-GPU run measures the headline step only, so its GPUs are not held for
    # minutes of untimed work
    if not args.core_only and world == 1:
        extras["precision_interior"] = precision_leg(cr, scenes, rank, world, args)
        extras["table3_sweep"] = sweep_leg(cr, S, cam, out, stream, rank, world)
        # the paper sweeps an indoor scene (Sibenik): the same sweep on the interior, 4 bounces
        si = scenes.interior()
        Si = cr.Scene(si)
        outi = torch.empty((si.camera.height, si.camera.width, 3), dtype=torch.float32, device="cuda")
        extras["table3_sweep_interior"] = sweep_leg(cr, Si, si.camera, outi, stream, rank, world, bounces=4)
        Si.close()
        extras["next_event_estimation"] = nee_leg(cr, scenes, rank, args)
        extras["transmission"] = transmission_leg(cr, scenes, rank, args)
        extras["quality"] = quality_leg(cr, S, cam, stream, results)
        # the indoor stand-in, closer to the paper's Table 2 scenes (its 4 bounces)
        si = scenes.interior()
        Si = cr.Scene(si)
        extras["quality_interior"] = quality_leg(cr, Si, si.camera, stream, results, bounces=4)
        Si.close()
        if not args.no_batched:
            extras["batched"] = batched_leg(cr, scenes, rank, args)
        if not args.no_serving and rank == 0:
            extras["serving"] = serving_leg(cr, scenes, args)

    if rank != 0:
        return
    R = results[modes[0]]
    # Roofline of the secondary trace kernel (k_trace_bvh2): the algorithmic node + triangle
    # bytes per secondary ray (32 ray + 4 queue + 8 hit + 64 per node visit + 48 per triangle
    # test, visits and tests from the counting pass) times the rays of one launch, over the
    # launch's CUDA-event time, against the measured HBM copy bandwidth (the headline) and
    # the measured L2 read roof.  Above the HBM roof means caches serve node fetches again
    # (coherence); the DRAM traffic the kernel really causes is the "traffic" key (ncu).
    # ncu shows the kernel bound by instruction issue (7-8 active lanes per warp
    # instruction), so the issue and FP32-ALU roofs are reported beside it.
    # With "+bvh8q" ("+bvh4") first, the figures describe k_trace_bvh8 (k_trace_bvh4) instead:
    # 80 B and 8 box tests (112 B and 4) per node visit, and no ncu-derived keys (the committed
    # summary is the BVH2 kernel's).
    layout0 = parse(modes[0])[3]
    plain = layout0 == cr.CR_BVH2
    node_b = {cr.CR_BVH2: 64, cr.CR_BVH8Q: 80, cr.CR_BVH4: 112}
    boxes = {cr.CR_BVH2: 2, cr.CR_BVH8Q: 8, cr.CR_BVH4: 4}
    launches = BOUNCES
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count  # cudaDevAttrMultiProcessorCount

    def node_bytes_per_ray(res, layout=cr.CR_BVH2):
        return trace_bytes_per_ray(res["nodes_per_ray"], res["tris_per_ray"], node_b[layout])

    rays_per_launch = R["secondary_rays_per_step"] / launches
    ms_per_launch = R["ms_trace_secondary"] / launches
    ops_per_ray = boxes[layout0] * 24 * R["nodes_per_ray"] + 40 * R["tris_per_ray"]
    achieved_ops = ops_per_ray * rays_per_launch / (ms_per_launch / 1e3) / 1e12
    clk = (clocks or {}).get("sm_mhz") or 2070.0
    peak_ops = n_sm * 128 * clk * 1e6 / 1e12
    bytes_per_ray = node_bytes_per_ray(R, layout0)
    achieved = bytes_per_ray * rays_per_launch / (ms_per_launch / 1e3) / 1e9
    peak, peak_kind = load_peaks()
    traffic = profile_traffic() if plain else None
    l2_gbs = l2_read_bandwidth(cr)
    # every mode's node-byte rate on the same roof (trace-only secondary rays/s x its own bytes
    # per ray), and its ratio to independent sampling's: the coherence gain read off one roof
    per_mode = {}
    for m in modes:
        lay = parse(m)[3]
        ach_m = node_bytes_per_ray(results[m], lay) * results[m]["trace_mrays"] * 1e6 / 1e9
        per_mode[m] = {"achieved": round(ach_m, 1), "frac": round(ach_m / peak, 4),
                       "bytes_per_ray": round(node_bytes_per_ray(results[m], lay), 1)}
    if "independent" in per_mode:
        for m in per_mode:
            per_mode[m]["frac_vs_independent"] = round(per_mode[m]["frac"] / per_mode["independent"]["frac"], 4)
    line = {
        "metric": METRIC, "value": round(R["mrays"], 2), "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(R["ms_per_step"], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "mode": modes[0], "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world} (frames per rank)", "timing": "CUDA events on the render stream"},
        "clocks": clocks,
        "e2e": {"value": round(e2e_rays / e2e["pipelined"] / 1e6, 2), "unit": "Mrays/s",
                "h2d_bytes_per_step": h2d_step, "d2h_bytes_per_step": cam.width * cam.height * 12,
                "timing": "host clock over the steps; each step's image copied to page-locked host memory on a "
                          "side stream while the next step renders (double-buffered), all copies inside the region; "
                          "no L2 flush between steps (the device-timed value flushes)",
                "sync_value": round(e2e_rays / e2e["sync"] / 1e6, 2),
                "sync_timing": "cr_render_ex into page-locked host memory, one synchronous call per step"},
        "gpu_launches": int(R["launches_per_step"] * args.steps),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": f"k_trace_{ {cr.CR_BVH2: 'bvh2', cr.CR_BVH8Q: 'bvh8', cr.CR_BVH4: 'bvh4'}[layout0]} (secondary rays)",
                     "bytes_per_ray": round(bytes_per_ray, 1), "rays_per_launch": round(rays_per_launch),
                     "ms_per_launch": round(ms_per_launch, 5),
                     "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_kind})",
                     "note": "algorithmic node+triangle bytes per launch / CUDA-event launch time; mostly served by "
                             "L1/L2, the DRAM bytes ncu counts per launch are 'traffic'",
                     "modes": per_mode},
        "roofline_alu": {"achieved": round(achieved_ops, 3), "peak": round(peak_ops, 2),
                         "unit": "TOP/s (FP32 ALU operations)", "frac": round(achieved_ops / peak_ops, 4),
                         "ops_per_ray": round(ops_per_ray, 1),
                         "peak_source": f"{n_sm} SMs (device attribute) x 128 FP32 lanes x {clk:.0f} MHz (sampled)"},
        "roofline_issue": issue_roof(R, clk, n_sm) if plain else None,
        "roofline_l2": {"achieved": round(achieved, 1), "peak": round(l2_gbs, 1), "unit": "GB/s",
                        "frac": round(achieved / l2_gbs, 4),
                        "peak_source": "cr_measure_l2_read: read-only kernel over an L2-resident 48 MB buffer, CUDA events",
                        "note": "algorithmic node+triangle bytes against the L2 roof; < 1 means L1 hits carry the rest"},
        "trace_only_mrays": round(R["trace_mrays"], 2),
        "stages_ms": {k: round(R[k], 4) for k in ("ms_trace_primary", "ms_trace_secondary", "ms_shade", "ms_compact",
                                                   "ms_sort", "ms_raygen", "ms_accum")},
        "stages_note": "trace stages from the timed steps; the others from 3 untimed steps with events between all stages",
        "comparators": {m: {"mrays": round(results[m]["mrays"], 2), "trace_only_mrays": round(results[m]["trace_mrays"], 2),
                            "ms_per_step": round(results[m]["ms_per_step"], 4),
                            "nodes_per_ray": round(results[m]["nodes_per_ray"], 2),
                            "tris_per_ray": round(results[m]["tris_per_ray"], 2),
                            "ms_sort": round(results[m]["ms_sort"], 4)}
                        for m in modes if m != "direction_reuse"},
        "secondary_rays_per_step": int(R["secondary_rays_per_step"]),
    }
    if "morton_sort" in results:
        # the comparator's ray sort (key kernel + three radix passes, per step): algorithmic bytes
        # per key = key kernel 38 in (queue 4, ray 32, scene 2) and 12 out (key, value, value
        # copy), then 3 passes x (8 in + 8 out) = 98, against the measured HBM copy bandwidth
        rm = results["morton_sort"]
        keys = rm["secondary_rays_per_step"]
        gbs = keys * 98 / (rm["ms_sort"] / 1e3) / 1e9 if rm["ms_sort"] > 0 else None
        line["sort_roofline"] = {"ms_per_step": round(rm["ms_sort"], 4), "keys_per_step": int(keys),
                                 "bytes_per_key": 98, "achieved": None if gbs is None else round(gbs, 1),
                                 "peak": peak, "unit": "GB/s", "frac": None if gbs is None else round(gbs / peak, 4),
                                 "share_of_step": round(rm["ms_sort"] / rm["ms_per_step"], 4),
                                 "timing": "stage events of 3 untimed steps (events between all stages)"}
    line.update(extras)
    if not args.no_cpu_baseline and world == 1:  # the oracle's rate is a single-GPU context figure
        v, thr, sample, dt = cpu_oracle_rate(sc, args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "Mrays/s", "cores": thr, "kind": "oracle",
                                "sample": sample}
        if not args.core_only:
            # the oracle on the other workloads (context): tiny in full, the interior at 1 spp
            # on a sample of tiles (a 16-spp render takes 16 times as long)
            extra = {}
            for name, scn, b in (("tiny", scenes.tiny(), 1), ("interior", scenes.interior(), 4)):
                v2, thr2, sample2, dt2 = cpu_oracle_rate(scn, 4.0, bounces=b)
                extra[name] = {"mrays": round(v2, 4), "cores": thr2, "sample": sample2, "seconds": round(dt2, 2)}
            line["cpu_baseline"]["other_workloads"] = extra
    print(json.dumps(line), flush=True)


def trace_bytes_per_ray(nodes_per_ray: float, tris_per_ray: float, node_bytes: int = 64) -> float:
    """Algorithmic bytes one secondary ray moves through the trace kernel: its ray record
    (32 B), the queue entry (4 B) and the hit (8 B), every node visited (64 B for a BVH2
    node, 80 for BVH8-Q, 112 for BVH4) and every triangle tested (48 B)."""
    return 32 + 4 + 8 + node_bytes * nodes_per_ray + 48 * tris_per_ray


def issue_roof(R, clk, n_sm):
    """The trace kernel's binding roof (ncu: issue-bound): warp instructions per second
    against one instruction per scheduler per clock (n_sm SMs x 4 schedulers).  Instructions
    per ray come from the committed ncu capture; the ray rate is this run's."""
    ipr = profile_traffic("warp_instructions_per_ray")
    peak = n_sm * 4 * clk * 1e6 / 1e12
    if ipr is None:
        return {"achieved": None, "peak": round(peak, 3), "unit": "T warp instructions/s", "frac": None}
    ach = ipr * R["trace_mrays"] * 1e6 / 1e12
    return {"achieved": round(ach, 3), "peak": round(peak, 3), "unit": "T warp instructions/s",
            "frac": round(ach / peak, 4), "instructions_per_ray": ipr,
            "source": "warp instructions per ray from profiles/k_trace_bvh2.landscape.txt x this run's trace-only rate"}


def l2_read_bandwidth(cr, mb=48, reps=100):
    """L2 roof of the roofline: GB/s read by the library's read-only probe kernel over an
    L2-resident buffer (measured, not a datasheet figure)."""
    return cr.cr_measure_l2_read(mb << 20, reps)


def _timed_renders(cr, S, cam, out, stream, steps, warmup, frame0=0, **kw):
    """Device time (ms, summed) and secondary rays of ``steps`` renders after ``warmup``."""
    import torch
    spp = kw.pop("spp", SPP)
    bounces = kw.pop("bounces", BOUNCES)
    mode = kw.pop("mode", "direction_reuse")
    tile = kw.pop("tile", TILE)
    extra_flags = kw.pop("extra_flags", 0)
    ms = tr = 0.0
    sec = 0
    for i in range(warmup + steps):
        st = cr.cr_stats()
        o = cr.make_opts(frame_base=frame0 + i, flags=cr.CR_OPT_STATS_TRACES | extra_flags, stream=stream, stats=st,
                         **kw)
        cr.cr_render_ex(S.handle, cam, spp, bounces, mode, tile[0], tile[1], out, o)
        if i >= warmup:
            d = st.as_dict()
            ms += d["ms_total"]
            tr += d["ms_trace_secondary"]
            sec += d["secondary_rays"]
    torch.cuda.synchronize()
    return ms, tr, sec


def precision_leg(cr, scenes, rank, world, args):
    """Interior (1280x720, 512,014 triangles, 16 spp, 4 bounces, direction reuse): FP32 BVH2
    vs the 8-bit quantised BVH8-Q and the FP32 4-wide BVH4; the images must be identical bit
    for bit."""
    import torch
    sc = scenes.interior()
    S8 = cr.Scene(sc, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q | cr.CR_BVH4)
    cam = sc.camera
    out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    res = {"workload": "interior 1280x720, 2,000 UV spheres + room + ceiling light (512,014 tris), 16 spp, "
                       "4 bounces, direction_reuse 8x8 K=8", "scene_bytes": S8.info["device_bytes"]}
    imgs = {}
    for name, bvh in (("bvh2", cr.CR_BVH2), ("bvh8q", cr.CR_BVH8Q), ("bvh4", cr.CR_BVH4)):
        ms, tr, sec = _timed_renders(cr, S8, cam, out, stream, 3, 2, frame0=rank * 100, spp=16, bounces=4, k=K,
                                     bvh=bvh)
        ms = aggregate(ms, "max")
        sec = aggregate(sec, "sum")
        res[name] = {"mrays": round(sec / ms / 1e3, 2), "trace_only_mrays": round(sec / aggregate(tr, "max") / 1e3, 2),
                     "ms_per_render": round(ms / 3, 3)}
        o = cr.make_opts(k=K, frame_base=0, bvh=bvh, stream=stream)
        cr.cr_render_ex(S8.handle, cam, 16, 4, "direction_reuse", 8, 8, out, o)
        imgs[name] = out.clone()
    res["images_bit_identical"] = bool(torch.equal(imgs["bvh2"], imgs["bvh8q"]) and torch.equal(imgs["bvh2"], imgs["bvh4"]))
    res["nodes"] = {"bvh2": S8.info["n_nodes2"], "bvh8q": S8.info["n_nodes8"], "bvh4": S8.info["n_nodes4"]}
    S8.close()
    return res


def nee_leg(cr, scenes, rank, args):
    """Next-event estimation on the interior (640x360, 512,014 triangles, small ceiling light,
    4 bounces): ray throughput with shadow rays, and MSE at equal device time against a
    2048-spp independent + NEE reference (both estimators have the same mean)."""
    import torch
    sc = scenes.interior(width=640, height=360)
    S = cr.Scene(sc)
    cam = sc.camera
    stream = torch.cuda.current_stream().cuda_stream
    img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    ref = torch.zeros_like(img)
    B = 4

    def render(spp, mode, nee, frame, stats=None):
        # nee: 0 off, 1 one light sample per pixel, 2 one light point per reuse group
        o = cr.make_opts(k=K, frame_base=frame, stream=stream, stats=stats,
                         flags=(cr.CR_OPT_NEE if nee else 0) | (cr.CR_OPT_NEE_SHARED if nee == 2 else 0) |
                         (cr.CR_OPT_STATS_TRACES if stats is not None else 0))
        cr.cr_render_ex(S.handle, cam, spp, B, mode, TILE[0], TILE[1], img, o)

    n_ref = 2048
    for c in range(0, n_ref, 256):
        render(256, "independent", 1, 5_000_000 + c)
        ref += img
    ref /= n_ref // 256
    torch.cuda.synchronize()
    out = {"workload": "interior 640x360, 512,014 tris, 4 bounces, 8x8 K=8", "reference_spp": n_ref,
           "budgets_s": [0.05, 0.25], "modes": {}}
    for mode, nee in (("direction_reuse", 0), ("direction_reuse", 1), ("direction_reuse", 2), ("independent", 0),
                      ("independent", 1)):
        if True:
            ms = sec = shadow = tsh = 0.0
            for i in range(5):
                st = cr.cr_stats()
                render(1, mode, nee, rank * 100 + i, st)
                if i >= 2:
                    d = st.as_dict()
                    ms += d["ms_total"]
                    sec += d["secondary_rays"]
                    shadow += d["shadow_rays"]
                    tsh += d["ms_trace_shadow"]
            ms_spp = ms / 3
            row = {"ms_per_spp": round(ms_spp, 4), "mrays_incl_shadow": round((sec + shadow) / ms / 1e3, 1),
                   "secondary_rays_per_spp": int(sec / 3), "shadow_rays_per_spp": int(shadow / 3), "mse": [], "spp": []}
            if nee:
                row["shadow_trace_mrays"] = round(shadow / tsh / 1e3, 1) if tsh > 0 else None
            for T in out["budgets_s"]:
                spp = max(1, int(T * 1e3 / ms_spp))
                render(spp, mode, nee, 0)
                row["mse"].append(float(((img - ref) ** 2).mean()))
                row["spp"].append(spp)
            out["modes"][mode + ("", "+nee", "+nee_shared")[nee]] = row
    S.close()
    return out


def transmission_leg(cr, scenes, rank, args):
    """Transmission materials (Sec. 6 future work): 1M-triangle soup with 35/25/15/10/15
    Lambert/translucent/GGX/mirror/dielectric triangles, 1024x1024, 1 spp, 3 bounces, 8x8
    K=8.  Translucent points join the diffuse class (lower-hemisphere lobe), so groups mixing
    them with Lambert points still share one direction."""
    import numpy as np
    import torch
    sc = scenes.tiny(seed=9, n_soup=1_000_000, width=1024, height=1024, material_mix="transmissive")
    S = cr.Scene(sc)
    cam = sc.camera
    out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    res = {"workload": "soup 1M tris, transmissive mix, 1024x1024, 1 spp, B=3, 8x8 K=8"}
    for mode in ("direction_reuse", "independent"):
        ms, tr, sec = _timed_renders(cr, S, cam, out, stream, 5, 2, frame0=rank * 100, bounces=3, mode=mode, k=K)
        res[mode] = {"mrays": round(sec / ms / 1e3, 1), "trace_only_mrays": round(sec / tr / 1e3, 1)}
    res["trace_ratio_reuse_over_independent"] = round(res["direction_reuse"]["trace_only_mrays"] /
                                                      res["independent"]["trace_only_mrays"], 3)
    dbg, bufs = cr.debug_buffers(cam.width, cam.height, 1)
    o = cr.make_opts(k=K, frame_base=0, stream=stream, debug=dbg)
    cr.cr_render_ex(S.handle, cam, 1, 1, "direction_reuse", TILE[0], TILE[1], out, o)
    cls = bufs["cls"][0].cpu().numpy()
    cat = bufs["cat"][0].cpu().numpy()
    alive = cls > 0
    res["bounce1_classes"] = {"lambert": round(float((cls == 1).sum() / alive.sum()), 3),
                              "translucent": round(float((cls == 3).sum() / alive.sum()), 3),
                              "glossy_specular": round(float((cls == 2).sum() / alive.sum()), 3)}
    res["bounce1_categories"] = {name: round(float((cat[alive] == c).mean()), 3)
                                 for c, name in ((1, "diffuse"), (2, "glossy"), (3, "hybrid"))}
    S.close()
    return res


def sweep_leg(cr, S, cam, out, stream, rank, world, bounces=None):
    """Tile (W,H) x group size K sweep (the analogue of Table 3): secondary trace-only
    Mrays/s of direction reuse and its ratio to independent sampling."""
    kb = {} if bounces is None else {"bounces": bounces}
    ms, tr, sec = _timed_renders(cr, S, cam, out, stream, 3, 1, mode="independent", k=K, **kb)
    base = sec / tr / 1e3
    rows = {}
    for tile in ((8, 8), (16, 8), (16, 16), (32, 8)):
        for k in (8, 16, 32, 64):
            ms, tr, sec = _timed_renders(cr, S, cam, out, stream, 3, 1, tile=tile, k=k, **kb)
            v = sec / tr / 1e3
            rows[f"{tile[0]}x{tile[1]}_K{k}"] = {"trace_only_mrays": round(v, 1), "ratio": round(v / base, 3),
                                                 "whole_step_mrays": round(sec / ms / 1e3, 1)}
    return {"independent_trace_only_mrays": round(base, 1), "direction_reuse": rows}


T975 = {2: 12.706, 3: 4.303, 4: 3.182, 5: 2.776, 6: 2.571, 7: 2.447, 8: 2.365}  # Student t, 97.5%, by n samples


def _mean_ci(xs):
    """Mean and the half-width of its 95% confidence interval (Student t)."""
    n = len(xs)
    m = sum(xs) / n
    if n < 2:
        return m, None
    sd = math.sqrt(sum((x - m) ** 2 for x in xs) / (n - 1))
    return m, T975.get(n, 1.96) * sd / math.sqrt(n)


def quality_leg(cr, S, cam, stream, results, bounces=None, seeds=5, budgets=(0.1, 0.5, 2.0)):
    """MSE at equal time (Sec. 5.2) against a 4096-spp independent reference: for each mode
    and each of `seeds` Philox keys, samples accumulate progressively (frame_base continues)
    until each budget of device time per mode is spent; the mean MSE over keys and its 95%
    confidence interval per budget.  PSNR at 128 spp per key (the analogue of Table 2).  The
    fraction of live pixels in each group category per bounce (Sec. 3.2).  target_met: a mode
    with more whole-step secondary Mrays/s than both comparators and a lower mean MSE at
    every budget."""
    import torch
    B = bounces or BOUNCES
    ref = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    img = torch.empty_like(ref)
    part = torch.empty_like(ref)
    n_ref = 4096
    for ci, c in enumerate(range(0, n_ref, 256)):  # mean of 16 chunks of 256 samples
        o = cr.make_opts(k=K, seed=1000, frame_base=c, stream=stream)
        cr.cr_render_ex(S.handle, cam, 256, B, "independent", TILE[0], TILE[1], img, o)
        if ci == 0:
            ref.copy_(img)
        else:
            ref += img
    ref /= n_ref // 256
    torch.cuda.synchronize()
    peak = float(ref.max())
    out = {"reference_spp": n_ref, "reference": "independent sampling, Philox key 1000", "budgets_s": list(budgets),
           "seeds": seeds, "ci": "95%, Student t over the keys", "modes": {}}
    donor = cr.CR_OPT_HYBRID_DONOR
    variants = (("direction_reuse", "direction_reuse", 0), ("independent", "independent", 0),
                ("morton_sort", "morton_sort", 0), ("direction_reuse_hybrid_donor", "direction_reuse", donor))

    def render(spp, mode, flags, seed, frame, dst):
        o = cr.make_opts(k=K, seed=seed, frame_base=frame, stream=stream, flags=flags)
        cr.cr_render_ex(S.handle, cam, spp, B, mode, TILE[0], TILE[1], dst, o)

    for name, mode, vflags in variants:
        kw = {} if bounces is None else {"bounces": bounces}
        ms, tr, sec = _timed_renders(cr, S, cam, img, stream, 5, 2, mode=mode, extra_flags=vflags, **kw)
        ms_spp = ms / 5
        mrays = sec / (ms / 1e3) / 1e6
        row = {"ms_per_spp": round(ms_spp, 4), "whole_step_mrays": round(mrays, 1), "spp": [], "mse": [],
               "mse_ci95": [], "psnr_128spp_db": None}
        spps = [max(1, int(T * 1e3 / ms_spp)) for T in budgets]
        row["spp"] = spps
        per_budget = [[] for _ in budgets]
        psnr = []
        for seed in range(seeds):
            done = 0
            for bi, n in enumerate(spps):  # progressive: the next budget continues the frames
                if n > done:
                    render(n - done, mode, vflags, seed, done, part)
                    if done == 0:
                        img.copy_(part)
                    else:
                        img.mul_(done / n).add_(part, alpha=(n - done) / n)
                    done = n
                per_budget[bi].append(float(((img - ref) ** 2).mean()))
            render(128, mode, vflags, seed, 50_000, img)
            psnr.append(10 * math.log10(peak * peak / float(((img - ref) ** 2).mean())))
        for vals in per_budget:
            m, h = _mean_ci(vals)
            row["mse"].append(m)
            row["mse_ci95"].append(h)
        pm, ph = _mean_ci(psnr)
        row["psnr_128spp_db"] = round(pm, 3)
        row["psnr_128spp_ci95_db"] = None if ph is None else round(ph, 3)
        # bias estimate: a 1024-spp mean of the mode against the reference
        render(1024, mode, vflags, 0, 2_000_000, img)
        row["mse_1024spp"] = float(((img - ref) ** 2).mean())
        out["modes"][name] = row
    # the paper's target per mode: faster than both comparators and lower MSE at every budget
    comps = ("independent", "morton_sort")
    for name, row in out["modes"].items():
        if name in comps:
            continue
        faster = all(row["whole_step_mrays"] > out["modes"][c]["whole_step_mrays"] for c in comps)
        lower = all(row["mse"][i] < out["modes"][c]["mse"][i] for c in comps for i in range(len(budgets)))
        separated = all(row["mse"][i] + (row["mse_ci95"][i] or 0) < out["modes"][c]["mse"][i]
                        - (out["modes"][c]["mse_ci95"][i] or 0) for c in comps for i in range(len(budgets)))
        row["target_met"] = bool(faster and lower)
        row["faster_than_both"] = bool(faster)
        row["lower_mse_than_both"] = bool(lower)
        row["lower_mse_ci_separated"] = bool(separated)
    out["category_fractions"] = category_fractions(cr, S, cam, stream, B)
    return out


def category_fractions(cr, S, cam, stream, B):
    """Fraction of the live pixels whose reuse group is diffuse / glossy / hybrid at each
    bounce (Sec. 3.2), from one frame's per-bounce capture."""
    import torch
    dbg, bufs = cr.debug_buffers(cam.width, cam.height, B)
    img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    o = cr.make_opts(k=K, seed=0, frame_base=0, stream=stream, debug=dbg)
    cr.cr_render_ex(S.handle, cam, 1, B, "direction_reuse", TILE[0], TILE[1], img, o)
    torch.cuda.synchronize()
    rows = []
    for b in range(B):
        live = (bufs["flags"][b] & 1).bool()
        n = max(1, int(live.sum()))
        cat = bufs["cat"][b][live]
        rows.append({"bounce": b + 1, "live_pixels": n,
                     **{k: round(int((cat == v).sum()) / n, 4) for k, v in (("diffuse", 1), ("glossy", 2),
                                                                           ("hybrid", 3))}})
    return rows


def batched_leg(cr, scenes, rank, args):
    """64 jobs (sides uniform over 256..1024 in steps of 256, over the terrain, the interior and
    random soups of 1M and 4M triangles), 4 spp, 3 bounces, direction reuse: one wavefront per
    sample pass, CUDA-graph replay, tile shape / K / interleave / block from the autotuner.
    Compared with rendering the same jobs one at a time and with the untuned default."""
    import numpy as np
    import torch
    rng = np.random.default_rng(21)
    world = {"terrain": scenes.landscape(), "interior": scenes.interior(), "soup1m": scenes.soup(31, 1_000_000),
             "soup4m": scenes.soup(32, 4_000_000)}
    S = {k: cr.Scene(v) for k, v in world.items()}
    names = list(world)
    specs = []
    for i in range(64):
        side = int(rng.choice([256, 512, 768, 1024]))
        specs.append((names[int(rng.integers(0, 4))], side, int(rng.integers(0, 1 << 30))))
    outs = [torch.empty((sd, sd, 3), dtype=torch.float32, device="cuda") for _, sd, _ in specs]

    def jobs_for(spp):
        js = []
        for (name, sd, seed), o in zip(specs, outs):
            c = world[name].camera
            cam = scenes.Camera(c.pos, c.look_at, c.up, c.vfov_deg, sd, sd)
            js.append(cr.make_job(S[name].handle, cam, o, spp=spp, max_bounces=3, mode="direction_reuse", seed=seed,
                                  frame_base=rank * 1000))
        return js

    jobs = jobs_for(4)
    opts = cr.make_batch_opts(tile=(8, 8), k=8)
    t0 = time.perf_counter()
    rep = cr.cr_batch_autotune(jobs_for(1), opts, allow_contiguous=True)
    tune_s = time.perf_counter() - t0
    res = {"workload": "64 jobs, sides {256,512,768,1024}^2, scenes {terrain 2.1M, interior 0.5M, soup 1M, soup 4M}, "
                       "4 spp, 3 bounces, direction_reuse",
           "pixels": int(sum(sd * sd for _, sd, _ in specs)),
           "autotune": {"seconds": round(tune_s, 1), "candidates": rep["n_candidates"],
                        "best": f"{opts.group_w}x{opts.group_h} K={opts.k} interleave={'lcg' if opts.interleave else 'contiguous'} block={opts.block} stack={opts.stack}",
                        "best_ms_spp1": round(rep["best_ms"], 3), "default_ms_spp1": round(rep["default_ms"], 3),
                        "quality_guard": {"probe_job": rep["probe_job"], "best_block_mse": rep["best_mse"],
                                          "default_block_mse": rep["default_mse"], "rejected": rep["n_rejected"],
                                          "measure": "MSE of 4x4-pixel block means against a 64-spp independent "
                                                     "reference; groupings above 1.1x the default's are not chosen"}}}
    variants = {"graph_autotuned": (opts, cr.CR_BATCH_GRAPH),
                "graph_default": (cr.make_batch_opts(tile=(8, 8), k=8), cr.CR_BATCH_GRAPH),
                "direct_autotuned": (opts, 0)}
    for name, (o, flags) in variants.items():
        oo = cr.make_batch_opts(tile=(o.group_w, o.group_h), k=o.k, interleave=bool(o.interleave), block=o.block,
                                flags=flags)
        b = cr.cr_batch_create(jobs, oo)
        cr.cr_batch_run(b)
        ms, sec, launches = [], 0, 0
        for _ in range(3):
            st = cr.cr_batch_run(b)
            ms.append(st["ms_total"])
            sec += st["secondary_rays"]
            launches = st["kernel_launches"]
        cr.cr_batch_destroy(b)
        res[name] = {"ms_per_batch": round(sum(ms) / 3, 2), "mrays": round(sec / sum(ms) / 1e3, 1),
                     "launches_per_batch": launches}
    # the same jobs rendered one at a time (one job per wavefront, no graph)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sec = 0
    ev0.record()
    for (name, sd, seed), o in zip(specs, outs):
        c = world[name].camera
        cam = scenes.Camera(c.pos, c.look_at, c.up, c.vfov_deg, sd, sd)
        st = cr.cr_stats()
        cr.cr_render_ex(S[name].handle, cam, 4, 3, "direction_reuse", opts.group_w, opts.group_h, o,
                        cr.make_opts(k=opts.k, interleave=bool(opts.interleave), block=opts.block, seed=seed,
                                     frame_base=rank * 1000, stream=stream, stats=st))
        sec += st.secondary_rays
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    res["one_at_a_time"] = {"ms_per_batch": round(ms, 2), "mrays": round(sec / ms / 1e3, 1)}
    for v in S.values():
        v.close()
    return res


EXPRESS_RAYS = 1 << 26  # ray steps (pixels x spp x (bounces + 1)) of the serving leg's express requests


def serving_leg(cr, scenes, args):
    """Poisson arrivals against six resident scenes (tiny, soups 1M/4M, interior, landscape,
    terrain 2236^2 = 9,990,450 triangles), sides log-uniform in [128, 2048] (multiples of
    16), spp in {1,4,16,64}, 1-4 bounces, host outputs; p50/p99 latency from submission to
    the result on the host, and throughput, for direction reuse + BVH8-Q, independent
    sampling + BVH2 and direction reuse + BVH2, the last also with the express lane (requests
    of at most EXPRESS_RAYS ray steps in a second, higher-priority wavefront)."""
    import numpy as np
    world = {"tiny": scenes.tiny(), "soup1m": scenes.soup(31, 1_000_000), "soup4m": scenes.soup(32, 4_000_000),
             "interior": scenes.interior(), "landscape": scenes.landscape(), "terrain": scenes.terrain()}
    S = {k: cr.Scene(v, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q) for k, v in world.items()}
    names = list(world)
    out = {"window_s": args.serve_window, "drain_s": args.serve_drain, "rates": list(args.serve_rates),
           "latency": "submission to the result on the host, over the requests completed by the end of the drain; "
                      "queue wait = admission - submission, render = completion - admission",
           "configs": {}}
    configs = (("reuse_bvh8q", "direction_reuse", cr.CR_BVH8Q, 0), ("independent_bvh2", "independent", cr.CR_BVH2, 0),
               ("reuse_bvh2", "direction_reuse", cr.CR_BVH2, 0),
               ("reuse_bvh2_express", "direction_reuse", cr.CR_BVH2, EXPRESS_RAYS))
    out["express_rays"] = EXPRESS_RAYS
    for cfg, mode, bvh, express in configs:
        if getattr(args, "serve_configs", None) and cfg not in args.serve_configs:
            continue
        rows = {}
        for lam in args.serve_rates:
            rng = np.random.default_rng(41 + int(lam))
            srv = cr.cr_server_create(48 << 30, tile=(8, 8), k=8, bvh=bvh, express_rays=express)
            t_next = 0.0
            arrivals = []
            while True:
                t_next += rng.exponential(1.0 / lam)
                if t_next > args.serve_window:
                    break
                arrivals.append(t_next)
            reqs = []
            t0 = time.perf_counter()
            for ta in arrivals:
                side = int(round(math.exp(rng.uniform(math.log(128), math.log(2048))) / 16) * 16)
                name = names[int(rng.integers(0, 6))]
                spp = int(rng.choice([1, 4, 16, 64]))
                B = int(rng.integers(1, 5))
                c = world[name].camera
                cam = scenes.Camera(c.pos, c.look_at, c.up, c.vfov_deg, side, side)
                host = np.empty((side, side, 3), np.float32)
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                jid = cr.cr_server_submit(srv, cr.make_job(S[name].handle, cam, host, spp=spp, max_bounces=B,
                                                           mode=mode, seed=int(rng.integers(0, 1 << 30))))
                reqs.append((jid, host))
            window_end_ms = args.serve_window * 1e3
            # drain: at rates the GPU sustains every request finishes; under overload the
            # backlog left after the drain is reported (and dropped with the server)
            done, t_drain = {}, time.perf_counter()
            while len(done) < len(reqs) and time.perf_counter() - t_drain < args.serve_drain:
                for jid, _ in reqs:
                    if jid not in done:
                        r = cr.cr_server_poll(srv, jid)
                        if r is not None:
                            done[jid] = r
                time.sleep(0.002)
            wall = time.perf_counter() - t0
            st = cr.cr_server_get_stats(srv)
            cr.cr_server_destroy(srv)
            js = list(done.values())
            lat = [j["latency_ms"] for j in js]
            wait = [j["t_admit_ms"] - j["t_submit_ms"] for j in js]
            rend = [j["t_done_ms"] - j["t_admit_ms"] for j in js]

            def pct(v, q):
                return round(float(np.percentile(v, q)), 1) if v else None

            t_first = min((j["t_submit_ms"] for j in js), default=0.0)
            rows[str(lam)] = {
                "arrivals": len(reqs), "completed": len(js),
                "completed_in_window": sum(1 for j in js if j["t_done_ms"] - t_first <= window_end_ms),
                "admitted_in_window": sum(1 for j in js if j["t_admit_ms"] - t_first <= window_end_ms),
                "unfinished_after_drain": len(reqs) - len(js),
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "queue_wait_p50_ms": pct(wait, 50), "queue_wait_p99_ms": pct(wait, 99),
                "render_p50_ms": pct(rend, 50), "render_p99_ms": pct(rend, 99),
                "wall_s": round(wall, 2), "mrays": round(st["secondary_rays"] / wall / 1e6, 1),
                "passes": st["passes"]}
        out["configs"][cfg] = rows
    for v in S.values():
        v.close()
    return out


def sort_only(args):
    """The Morton comparator's ray sort alone (cr_debug_sort) on N random 30-bit keys: mean
    device time of a sort over --sort-reps runs after one warm-up, as one JSON line."""
    import numpy as np
    import torch
    from paper_2310_07182_gb300 import binding as cr
    from paper_2310_07182_gb300 import build as crbuild
    crbuild.build()
    n = args.sort_keys
    rng = np.random.default_rng(1)
    keys = torch.from_numpy(rng.integers(0, 1 << 30, n, dtype=np.int64).astype(np.uint32).view(np.int32)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    cr.cr_debug_sort(keys, vals, reps=1)
    _, _, ms = cr.cr_debug_sort(keys, vals, reps=args.sort_reps)
    print(json.dumps({"sort_keys": n, "reps": args.sort_reps, "ms_per_sort": round(ms, 5),
                      "algorithmic_gbs": round(n * (8 + 12 + 3 * 16) / (ms * 1e-3) / 1e9, 1)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--core-only", action="store_true", help="skip the precision, sweep, quality, batched and serving legs")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--sort-keys", type=int, default=0, help="time the ray sort alone on this many keys and exit")
    ap.add_argument("--sort-reps", type=int, default=20)
    ap.add_argument("--serve-window", type=float, default=10.0, help="seconds of Poisson arrivals per rate")
    ap.add_argument("--serve-drain", type=float, default=5.0, help="seconds to wait for the requests after the window")
    ap.add_argument("--serve-rates", type=lambda x: [float(v) for v in x.split(",")], default=[20.0, 50.0, 100.0, 200.0])
    ap.add_argument("--serve-configs", type=lambda x: x.split(","), default=None,
                    help="serving configurations to run (default: all)")
    ap.add_argument("--scene", default="landscape", choices=["landscape", "interior"],
                    help="workload scene; the headline metric is the landscape's")
    ap.add_argument("--modes", default="direction_reuse,independent,morton_sort,world_reuse",
                    help="modes to time (the first is the headline); profiling runs use one")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    if args.sort_keys:
        sort_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
