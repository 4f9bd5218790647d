"""Thin ctypes binding of libcr.so (include/cr.h).

Each ``cr_*`` function here marshals its arguments and calls the C entry point of the same
name; every step of the path runs in the library's CUDA kernels.  PyTorch is used only for
device memory and streams: arrays may be numpy arrays (host) or torch tensors (host or
CUDA); CUDA tensors are passed by ``data_ptr()`` and the call runs on torch's current
stream unless a stream is given.

The library must have been built (``python -m paper_2310_07182_gb300.build`` or
``__graft_entry__.build()``); importing a function that needs it raises if libcr.so is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# CR_LIB selects another build of the library (the debug build, libcr_debug.so) for a process
LIB_PATH = os.environ.get("CR_LIB") or os.path.join(_PKG, "libcr.so")

CR_OK, CR_ERR_INVALID_ARG, CR_ERR_OOM, CR_ERR_CUDA, CR_ERR_TIMEOUT, CR_ERR_STACK_OVERFLOW, CR_ERR_BUSY, \
    CR_ERR_NOT_FOUND = range(8)
CR_MAT_LAMBERT, CR_MAT_GGX, CR_MAT_MIRROR, CR_MAT_EMITTER, CR_MAT_DIELECTRIC, CR_MAT_TRANSLUCENT = range(6)
CR_BVH2, CR_BVH8Q, CR_BVH4 = 1, 2, 4
CR_INDEPENDENT, CR_MORTON_SORT, CR_DIRECTION_REUSE, CR_WORLD_REUSE = 0, 1, 2, 3
CR_OPT_STATS, CR_OPT_COUNT, CR_OPT_NO_SYNC, CR_OPT_PERSISTENT, CR_OPT_SPECULATIVE = 1, 2, 4, 8, 16
CR_OPT_PACKET_PRIMARY, CR_OPT_PACKET_SECONDARY, CR_OPT_TWO_PHASE = 32, 64, 128
CR_OPT_NEE, CR_OPT_ANY_HIT, CR_OPT_HYBRID_DONOR, CR_OPT_NEE_SHARED = 256, 512, 1024, 2048
CR_OPT_STATS_TRACES = 4096
CR_OPT_ORDERED_QUEUES = 8192
CR_JOB_NEE, CR_JOB_HYBRID_DONOR, CR_JOB_NEE_SHARED = 1, 2, 4
MODES = {"independent": CR_INDEPENDENT, "morton_sort": CR_MORTON_SORT, "direction_reuse": CR_DIRECTION_REUSE,
         "world_reuse": CR_WORLD_REUSE}


class CrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cr status {status}: {msg}")
        self.status = status


class cr_material(C.Structure):
    _fields_ = [("type", C.c_uint32), ("albedo", C.c_float * 3), ("roughness", C.c_float),
                ("emission", C.c_float * 3)]


class cr_env(C.Structure):
    _fields_ = [("radiance", C.c_float * 3)]


class cr_scene_info(C.Structure):
    _fields_ = [("n_tri", C.c_uint32), ("n_mat", C.c_uint32), ("n_nodes2", C.c_uint32), ("depth2", C.c_uint32),
                ("n_nodes8", C.c_uint32), ("n_lights", C.c_uint32), ("device_bytes", C.c_uint64),
                ("build_ms", C.c_double), ("bounds_lo", C.c_float * 3), ("bounds_hi", C.c_float * 3),
                ("light_area", C.c_float), ("n_nodes4", C.c_uint32), ("depth4", C.c_uint32)]


class cr_camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class cr_stats(C.Structure):
    _fields_ = [("ms_total", C.c_double), ("ms_raygen", C.c_double), ("ms_trace_primary", C.c_double),
                ("ms_trace_secondary", C.c_double), ("ms_shade", C.c_double), ("ms_compact", C.c_double),
                ("ms_sort", C.c_double), ("ms_accum", C.c_double), ("primary_rays", C.c_uint64),
                ("secondary_rays", C.c_uint64), ("secondary_rays_b1", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("node_visits", C.c_uint64), ("tri_tests", C.c_uint64),
                ("shadow_rays", C.c_uint64), ("ms_trace_shadow", C.c_double), ("h2d_bytes", C.c_uint64),
                ("d2h_bytes", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cr_bvh_report(C.Structure):
    _fields_ = [("n_nodes2", C.c_uint32), ("depth2", C.c_uint32), ("n_nodes8", C.c_uint32), ("depth8", C.c_uint32),
                ("stack_bound8", C.c_uint32), ("covered2", C.c_uint32), ("covered8", C.c_uint32),
                ("violations2", C.c_uint32), ("violations8", C.c_uint32), ("pad", C.c_uint32),
                ("build_ms2", C.c_double), ("build_ms8", C.c_double), ("n_nodes4", C.c_uint32), ("depth4", C.c_uint32),
                ("stack_bound4", C.c_uint32), ("covered4", C.c_uint32), ("violations4", C.c_uint32),
                ("pad4", C.c_uint32)]


class cr_debug(C.Structure):
    _fields_ = [("prim", C.c_void_p), ("cat", C.c_void_p), ("cls", C.c_void_p), ("flags", C.c_void_p),
                ("local", C.c_void_p), ("world", C.c_void_p), ("ray", C.c_void_p), ("t", C.c_void_p),
                ("beta", C.c_void_p)]


class cr_job(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("camera", cr_camera), ("spp", C.c_uint32), ("max_bounces", C.c_uint32),
                ("mode", C.c_uint32), ("reuse_depth", C.c_uint32), ("seed", C.c_uint64), ("frame_base", C.c_uint32),
                ("flags", C.c_uint32), ("out_rgb", C.c_void_p), ("diffuse_roughness", C.c_float)]


class cr_batch_opts(C.Structure):
    _fields_ = [("group_w", C.c_uint32), ("group_h", C.c_uint32), ("k", C.c_uint32), ("interleave", C.c_uint32),
                ("bvh", C.c_uint32), ("block", C.c_uint32), ("flags", C.c_uint32), ("sort_key", C.c_uint32),
                ("stack", C.c_uint32), ("stream", C.c_void_p)]


class cr_tune_report(C.Structure):
    _fields_ = [("n_candidates", C.c_uint32), ("best_group_w", C.c_uint32), ("best_group_h", C.c_uint32),
                ("best_k", C.c_uint32), ("best_interleave", C.c_uint32), ("best_block", C.c_uint32),
                ("best_stack", C.c_uint32), ("best_ms", C.c_double), ("worst_ms", C.c_double), ("default_ms", C.c_double),
                ("best_mse", C.c_double), ("default_mse", C.c_double), ("n_rejected", C.c_uint32),
                ("probe_job", C.c_uint32)]


class cr_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("group_w", C.c_uint32), ("group_h", C.c_uint32), ("k", C.c_uint32),
                ("interleave", C.c_uint32), ("bvh", C.c_uint32), ("block", C.c_uint32),
                ("express_rays", C.c_uint32), ("pad", C.c_uint32)]


class cr_job_stats(C.Structure):
    _fields_ = [("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double),
                ("latency_ms", C.c_double), ("samples", C.c_uint32), ("pad", C.c_uint32),
                ("footprint_bytes", C.c_uint64)]


class cr_server_stats(C.Structure):
    _fields_ = [("jobs_submitted", C.c_uint64), ("jobs_done", C.c_uint64), ("passes", C.c_uint64),
                ("secondary_rays", C.c_uint64), ("kernel_launches", C.c_uint64), ("used_bytes", C.c_uint64),
                ("busy_ms", C.c_double), ("queued", C.c_uint32), ("active", C.c_uint32)]


class cr_render_opts(C.Structure):
    _fields_ = [("k", C.c_uint32), ("interleave", C.c_uint32), ("seed", C.c_uint64), ("frame_base", C.c_uint32),
                ("reuse_depth", C.c_uint32), ("bvh", C.c_uint32), ("block", C.c_uint32), ("flags", C.c_uint32),
                ("sort_key", C.c_uint32), ("stack", C.c_uint32), ("diffuse_roughness", C.c_float),
                ("stream", C.c_void_p), ("stats", C.POINTER(cr_stats)),
                ("debug", C.POINTER(cr_debug)), ("tile_begin", C.c_uint32), ("tile_end", C.c_uint32)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("cr_last_error", C.c_char_p, []),
    ("cr_version", C.c_char_p, []),
    ("cr_scene_create", C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                  C.c_uint32, C.POINTER(C.c_void_p)]),
    ("cr_scene_destroy", C.c_int, [C.c_void_p]),
    ("cr_scene_get_info", C.c_int, [C.c_void_p, C.POINTER(cr_scene_info)]),
    ("cr_render_opts_default", C.c_int, [C.POINTER(cr_render_opts)]),
    ("cr_render", C.c_int, [C.c_void_p, C.POINTER(cr_camera), C.c_uint32, C.c_uint32, C.c_int, C.c_uint32,
                            C.c_uint32, C.c_void_p]),
    ("cr_render_ex", C.c_int, [C.c_void_p, C.POINTER(cr_camera), C.c_uint32, C.c_uint32, C.c_int, C.c_uint32,
                               C.c_uint32, C.c_void_p, C.POINTER(cr_render_opts)]),
    ("cr_trace_rays", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                C.POINTER(cr_render_opts)]),
    ("cr_debug_groups", C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                                  C.c_uint32, C.c_void_p]),
    ("cr_debug_philox", C.c_int, [C.c_uint64, C.c_void_p, C.c_uint32, C.c_void_p]),
    ("cr_debug_sample", C.c_int, [C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    ("cr_batch_create", C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(cr_batch_opts), C.POINTER(C.c_void_p)]),
    ("cr_batch_run", C.c_int, [C.c_void_p, C.POINTER(cr_stats)]),
    ("cr_batch_destroy", C.c_int, [C.c_void_p]),
    ("cr_batch_device_bytes", C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(cr_batch_opts), C.POINTER(C.c_uint64)]),
    ("cr_batch_autotune", C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.POINTER(cr_batch_opts),
                                    C.POINTER(cr_tune_report)]),
    ("cr_server_create", C.c_int, [C.POINTER(cr_server_opts), C.POINTER(C.c_void_p)]),
    ("cr_server_submit", C.c_int, [C.c_void_p, C.POINTER(cr_job), C.POINTER(C.c_uint64)]),
    ("cr_server_poll", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(cr_job_stats)]),
    ("cr_server_wait", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint32, C.POINTER(cr_job_stats)]),
    ("cr_server_get_stats", C.c_int, [C.c_void_p, C.POINTER(cr_server_stats)]),
    ("cr_server_destroy", C.c_int, [C.c_void_p]),
    ("cr_debug_bvh_check", C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.POINTER(cr_bvh_report)]),
    ("cr_trace_rays_static", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    ("cr_measure_l2_read", C.c_int, [C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]),
    ("cr_debug_sort", C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_double)]),
]
CR_TRACE_STATIC_MAX_RAYS = 65536


def exported_names():
    return [n for n, _, _ in _SIGS]


def lib():
    """Load libcr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcr.so not built ({LIB_PATH}); run paper_2310_07182_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != CR_OK:
        raise CrError(status, lib().cr_last_error().decode())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


def _current_stream(tensors=()):
    for t in tensors:
        if hasattr(t, "is_cuda") and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


# ---------------------------------------------------------------------------------------
# Entry points with the ABI's names.
def cr_version() -> str:
    return lib().cr_version().decode()


def cr_scene_create(tri_xyz, tri_mat, mat_type, mat_params, env=(0.0, 0.0, 0.0), bvh_flags=CR_BVH2):
    """Build and upload a scene; returns the opaque handle (an int)."""
    tri_xyz = np.ascontiguousarray(tri_xyz, dtype=np.float32).reshape(-1, 9)
    tri_mat = np.ascontiguousarray(tri_mat, dtype=np.uint32)
    mat_type = np.asarray(mat_type, dtype=np.uint32)
    mat_params = np.asarray(mat_params, dtype=np.float32).reshape(-1, 7)
    mats = (cr_material * len(mat_type))()
    for i, (t, p) in enumerate(zip(mat_type, mat_params)):
        mats[i].type = int(t)
        mats[i].albedo[:] = [float(v) for v in p[0:3]]
        mats[i].roughness = float(p[3])
        mats[i].emission[:] = [float(v) for v in p[4:7]]
    e = cr_env((C.c_float * 3)(*[float(v) for v in env]))
    out = C.c_void_p()
    _check(lib().cr_scene_create(_ptr(tri_xyz), tri_xyz.shape[0], _ptr(tri_mat), C.addressof(mats), len(mat_type),
                                 C.addressof(e), bvh_flags, C.byref(out)))
    return out.value


def cr_scene_destroy(handle):
    _check(lib().cr_scene_destroy(handle))


def cr_scene_get_info(handle) -> dict:
    info = cr_scene_info()
    _check(lib().cr_scene_get_info(handle, C.byref(info)))
    d = {k: getattr(info, k) for k, _ in info._fields_}
    d["bounds_lo"] = list(info.bounds_lo)
    d["bounds_hi"] = list(info.bounds_hi)
    return d


def make_camera(cam) -> cr_camera:
    return cr_camera((C.c_float * 3)(*cam.pos), (C.c_float * 3)(*cam.look_at), (C.c_float * 3)(*cam.up),
                     float(cam.vfov_deg), int(cam.width), int(cam.height))


SORT_KEYS = {"two_point": 0, "origin": 1, "reis": 2, "costa": 3, "aila_compact": 4, "hierarchy_cut": 5}


def make_opts(k=0, interleave=True, seed=0, frame_base=0, reuse_depth=0, bvh=CR_BVH2, block=0, flags=0,
              stream=None, stats=None, debug=None, sort_key=0, stack=0, diffuse_roughness=0.0,
              tiles=None) -> cr_render_opts:
    o = cr_render_opts()
    _check(lib().cr_render_opts_default(C.byref(o)))
    o.k, o.interleave, o.seed, o.frame_base = k, int(interleave), seed, frame_base
    o.reuse_depth, o.bvh, o.block, o.flags = reuse_depth, bvh, block, flags
    o.sort_key = SORT_KEYS.get(sort_key, sort_key)
    o.stack = stack
    o.diffuse_roughness = float(diffuse_roughness)
    o.stream = stream
    if stats is not None:
        o.stats = C.pointer(stats)
    if debug is not None:
        o.debug = C.pointer(debug)
    if tiles is not None:
        o.tile_begin, o.tile_end = tiles
    return o


def cr_render(handle, cam, spp, max_bounces, mode, group_w, group_h, out_rgb):
    c = make_camera(cam)
    _check(lib().cr_render(handle, C.byref(c), spp, max_bounces, MODES.get(mode, mode), group_w, group_h,
                           _ptr(out_rgb)))
    return out_rgb


def cr_render_ex(handle, cam, spp, max_bounces, mode, group_w, group_h, out_rgb, opts: cr_render_opts | None):
    c = make_camera(cam)
    if opts is not None and opts.stream is None:
        opts.stream = _current_stream([out_rgb])
    _check(lib().cr_render_ex(handle, C.byref(c), spp, max_bounces, MODES.get(mode, mode), group_w, group_h,
                              _ptr(out_rgb), C.byref(opts) if opts is not None else None))
    return out_rgb


def cr_trace_rays(handle, rays, skip, prim, t, opts: cr_render_opts | None = None):
    n = rays.shape[0]
    if opts is not None and opts.stream is None:
        opts.stream = _current_stream([rays, prim, t])
    _check(lib().cr_trace_rays(handle, _ptr(rays), _ptr(skip), n, _ptr(prim), _ptr(t),
                               C.byref(opts) if opts is not None else None))


CR_BATCH_GRAPH = 1


def make_job(scene_handle, cam, out, spp=1, max_bounces=1, mode="direction_reuse", reuse_depth=0, seed=0,
             frame_base=0, nee=False, hybrid_donor=False, nee_shared=False, diffuse_roughness=0.0) -> cr_job:
    j = cr_job()
    j.flags = ((CR_JOB_NEE if nee else 0) | (CR_JOB_HYBRID_DONOR if hybrid_donor else 0)
               | (CR_JOB_NEE_SHARED if nee_shared else 0))
    j.scene = scene_handle
    j.camera = make_camera(cam)
    j.spp, j.max_bounces, j.mode, j.reuse_depth = spp, max_bounces, MODES.get(mode, mode), reuse_depth
    j.seed, j.frame_base = seed, frame_base
    j.out_rgb = _ptr(out)
    j.diffuse_roughness = float(diffuse_roughness)
    return j


def make_batch_opts(tile=(8, 8), k=0, interleave=True, bvh=CR_BVH2, block=0, flags=0, stream=None,
                    stack=0) -> cr_batch_opts:
    o = cr_batch_opts()
    o.group_w, o.group_h, o.k, o.interleave = tile[0], tile[1], k, int(interleave)
    o.bvh, o.block, o.flags, o.stack = bvh, block, flags, stack
    o.stream = stream
    return o


def _job_array(jobs):
    arr = (cr_job * len(jobs))(*jobs)
    return arr


def cr_batch_create(jobs, opts: cr_batch_opts):
    arr = _job_array(jobs)
    out = C.c_void_p()
    _check(lib().cr_batch_create(C.addressof(arr), len(jobs), C.byref(opts), C.byref(out)))
    return out.value


def cr_batch_run(handle, stats=True):
    st = cr_stats() if stats else None
    _check(lib().cr_batch_run(handle, C.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def cr_batch_destroy(handle):
    _check(lib().cr_batch_destroy(handle))


def cr_batch_device_bytes(jobs, opts: cr_batch_opts) -> int:
    arr = _job_array(jobs)
    v = C.c_uint64()
    _check(lib().cr_batch_device_bytes(C.addressof(arr), len(jobs), C.byref(opts), C.byref(v)))
    return v.value


def cr_batch_autotune(jobs, opts: cr_batch_opts, allow_contiguous=False) -> dict:
    arr = _job_array(jobs)
    rep = cr_tune_report()
    _check(lib().cr_batch_autotune(C.addressof(arr), len(jobs), int(allow_contiguous), C.byref(opts), C.byref(rep)))
    return {k: getattr(rep, k) for k, _ in rep._fields_}


def cr_server_create(hbm_budget, tile=(8, 8), k=0, interleave=True, bvh=CR_BVH2, block=0, express_rays=0):
    o = cr_server_opts(int(hbm_budget), tile[0], tile[1], k, int(interleave), bvh, block, int(express_rays), 0)
    out = C.c_void_p()
    _check(lib().cr_server_create(C.byref(o), C.byref(out)))
    return out.value


def cr_server_submit(handle, job: cr_job) -> int:
    jid = C.c_uint64()
    _check(lib().cr_server_submit(handle, C.byref(job), C.byref(jid)))
    return jid.value


def cr_server_poll(handle, job_id):
    """Returns the job's stats dict once done, None while it is queued or rendering."""
    js = cr_job_stats()
    st = lib().cr_server_poll(handle, job_id, C.byref(js))
    if st == CR_ERR_BUSY:
        return None
    _check(st)
    return {k: getattr(js, k) for k, _ in js._fields_}


def cr_server_wait(handle, job_id, timeout_ms=60000):
    js = cr_job_stats()
    _check(lib().cr_server_wait(handle, job_id, timeout_ms, C.byref(js)))
    return {k: getattr(js, k) for k, _ in js._fields_}


def cr_server_get_stats(handle) -> dict:
    st = cr_server_stats()
    _check(lib().cr_server_get_stats(handle, C.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def cr_server_destroy(handle):
    _check(lib().cr_server_destroy(handle))


def cr_measure_l2_read(nbytes=48 << 20, reps=100) -> float:
    """L2 read bandwidth (GB/s) of a read-only kernel over an L2-resident buffer."""
    v = C.c_double()
    _check(lib().cr_measure_l2_read(C.c_uint64(nbytes), reps, C.byref(v)))
    return v.value


def cr_debug_bvh_check(tri_xyz, flags=CR_BVH2 | CR_BVH8Q | CR_BVH4) -> dict:
    tri_xyz = np.ascontiguousarray(tri_xyz, dtype=np.float32).reshape(-1, 9)
    r = cr_bvh_report()
    _check(lib().cr_debug_bvh_check(_ptr(tri_xyz), tri_xyz.shape[0], flags, C.byref(r)))
    return {k: getattr(r, k) for k, _ in r._fields_}


def check_static_trace_args(rays, skip, prim, t) -> int:
    """Validate cr_trace_rays_static's buffers before they reach C, which sees only raw
    pointers and cannot check their lengths: rays a contiguous (n, 8) float32 tensor, prim
    int32 and t float32 (skip int32, or None) contiguous with at least n elements, all CUDA
    tensors of one device.  Returns n; raises TypeError or ValueError."""
    import torch
    named = [("rays", rays), ("prim", prim), ("t", t)] + ([("skip", skip)] if skip is not None else [])
    for name, x in named:
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"cr_trace_rays_static: {name} must be a torch tensor, not {type(x).__name__}")
        if not x.is_contiguous():
            raise ValueError(f"cr_trace_rays_static: {name} must be contiguous")
    if rays.dim() != 2 or rays.shape[1] != 8:
        raise ValueError(f"cr_trace_rays_static: rays must have shape (n, 8), not {tuple(rays.shape)}")
    n = int(rays.shape[0])
    want = {"rays": torch.float32, "prim": torch.int32, "t": torch.float32, "skip": torch.int32}
    for name, x in named:
        if x.dtype != want[name]:
            raise TypeError(f"cr_trace_rays_static: {name} must be {want[name]}, not {x.dtype}")
        if name != "rays" and x.numel() < n:
            raise ValueError(f"cr_trace_rays_static: {name} holds {x.numel()} elements, fewer than n = {n}")
    devs = {x.device for _, x in named}
    if any(not x.is_cuda for _, x in named) or len(devs) != 1:
        raise ValueError("cr_trace_rays_static: every buffer must be a CUDA tensor of one device, got "
                         + ", ".join(f"{name} on {x.device}" for name, x in named))
    return n


def cr_trace_rays_static(handle, rays, skip, prim, t, stream=None):
    """Allocation-free closest hits (see include/cr.h); the buffers are checked first."""
    n = check_static_trace_args(rays, skip, prim, t)
    if stream is None:
        stream = _current_stream([rays, prim, t])
    _check(lib().cr_trace_rays_static(handle, _ptr(rays), _ptr(skip), n, _ptr(prim), _ptr(t), stream))


def cr_debug_groups(width, height, group_w, group_h, interleave, seed, frame, out):
    _check(lib().cr_debug_groups(width, height, group_w, group_h, int(interleave), seed, frame, _ptr(out)))
    return out


def cr_debug_sort(keys, vals, reps=1):
    """The ray sort on caller keys (numpy or CUDA tensors of uint32/int32 keys and int32 values)
    -> (sorted keys, sorted values, mean ms per sort), outputs like the inputs."""
    n = int(keys.shape[0])
    if isinstance(keys, np.ndarray):
        keys = np.ascontiguousarray(keys).view(np.uint32) if keys.dtype.itemsize == 4 else keys.astype(np.uint32)
        vals = np.ascontiguousarray(vals, dtype=np.int32)
        ko, vo = np.empty(n, np.uint32), np.empty(n, np.int32)
    else:
        import torch
        ko, vo = torch.empty_like(keys), torch.empty(n, dtype=torch.int32, device=keys.device)
    ms = C.c_double()
    _check(lib().cr_debug_sort(_ptr(keys), _ptr(vals), n, reps, _ptr(ko), _ptr(vo), C.byref(ms)))
    return ko, vo, ms.value


def cr_debug_philox(seed, ctr, out):
    _check(lib().cr_debug_philox(seed, _ptr(ctr), ctr.shape[0], _ptr(out)))
    return out


def cr_debug_sample(kind, n, wo, u, param, wi, weight, valid):
    _check(lib().cr_debug_sample(kind, n, _ptr(wo), _ptr(u), _ptr(param), _ptr(wi), _ptr(weight), _ptr(valid)))


# ---------------------------------------------------------------------------------------
# Convenience layer.
class Scene:
    """Device-resident scene built from a ``scenes.Scene`` (or raw arrays)."""

    def __init__(self, sc, bvh_flags=CR_BVH2):
        self.src = sc
        self.handle = cr_scene_create(sc.tri_xyz, sc.tri_mat, sc.mat_type, sc.mat_params, sc.env, bvh_flags)
        self.info = cr_scene_get_info(self.handle)

    def close(self):
        if self.handle:
            cr_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cam=None, *, spp=1, max_bounces=1, mode="direction_reuse", tile=(8, 8), k=0, interleave=True,
               seed=0, frame_base=0, reuse_depth=0, out=None, stats=False, flags=0, block=0, bvh=CR_BVH2,
               debug=None, stream=None, sort_key=0, nee=False, stack=0, hybrid_donor=False, nee_shared=False,
               diffuse_roughness=0.0, tiles=None):
        """Render into ``out`` (torch CUDA tensor or numpy array of h x w x 3 float32; a new
        CUDA tensor by default).  Returns (out, stats dict or None)."""
        import torch
        cam = cam or self.src.camera
        if out is None:
            out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
        st = cr_stats() if stats else None
        o = make_opts(k=k, interleave=interleave, seed=seed, frame_base=frame_base, reuse_depth=reuse_depth, bvh=bvh,
                      block=block, flags=flags | (CR_OPT_STATS if stats else 0) | (CR_OPT_NEE if nee else 0)
                      | (CR_OPT_HYBRID_DONOR if hybrid_donor else 0) | (CR_OPT_NEE_SHARED if nee_shared else 0),
                      stream=stream, stats=st, debug=debug, sort_key=sort_key, stack=stack,
                      diffuse_roughness=diffuse_roughness, tiles=tiles)
        cr_render_ex(self.handle, cam, spp, max_bounces, mode, tile[0], tile[1], out, o)
        return out, (st.as_dict() if st is not None else None)

    def trace(self, rays, skip=None, *, bvh=CR_BVH2, flags=0, block=0, stats=False, any_hit=False):
        """Closest hits of (n, 8) rays (torch CUDA tensor or numpy) -> (prim, t[, stats]).
        any_hit: visibility only (some occluder before tmax, or -1)."""
        flags |= CR_OPT_ANY_HIT if any_hit else 0
        import torch
        n = rays.shape[0]
        dev = rays.device if isinstance(rays, torch.Tensor) and rays.is_cuda else None
        if dev is not None:
            prim = torch.empty(n, dtype=torch.int32, device=dev)
            t = torch.empty(n, dtype=torch.float32, device=dev)
        else:
            prim = np.empty(n, dtype=np.int32)
            t = np.empty(n, dtype=np.float32)
        st = cr_stats() if stats else None
        o = make_opts(bvh=bvh, flags=flags, block=block, stats=st)
        cr_trace_rays(self.handle, rays, skip, prim, t, o)
        return (prim, t, st.as_dict()) if stats else (prim, t)


def debug_buffers(width, height, max_bounces, device="cuda", replay=False):
    """Allocate (and pre-fill) the per-bounce capture buffers; returns (cr_debug, dict of tensors).
    replay=True adds the replay capture (ray, t, beta of every trace)."""
    import torch
    npx = width * height
    B = max_bounces
    bufs = dict(prim=torch.full((B + 1, npx), -2, dtype=torch.int32, device=device),
                cat=torch.full((B, npx), 255, dtype=torch.uint8, device=device),
                cls=torch.zeros((B, npx), dtype=torch.uint8, device=device),
                flags=torch.zeros((B, npx), dtype=torch.uint8, device=device),
                local=torch.zeros((B, npx, 3), dtype=torch.float32, device=device),
                world=torch.zeros((B, npx, 3), dtype=torch.float32, device=device))
    names = ["prim", "cat", "cls", "flags", "local", "world"]
    if replay:
        bufs.update(ray=torch.zeros((B + 1, npx, 8), dtype=torch.float32, device=device),
                    t=torch.full((B + 1, npx), float("nan"), dtype=torch.float32, device=device),
                    beta=torch.zeros((B + 1, npx, 4), dtype=torch.float32, device=device))
        names += ["ray", "t", "beta"]
    d = cr_debug(*[bufs[k].data_ptr() for k in names])
    return d, bufs
