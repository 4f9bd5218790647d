"""CPU oracle for the direction-reuse path tracer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It wraps ``oracle.c`` (plain C, built with gcc) through ctypes and shares no
code with the CUDA library; both sides only consume the arrays produced by
``paper_2310_07182_gb300.scenes``.

``render`` parallelises over tile ranges with Python threads: each thread calls the
single-threaded C routine on a disjoint range of tiles (ctypes releases the GIL), so the
result does not depend on the thread count.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

INDEPENDENT, MORTON_SORT, DIRECTION_REUSE, WORLD_REUSE = 0, 1, 2, 3
CAT_EMPTY, CAT_DIFFUSE, CAT_GLOSSY, CAT_HYBRID = 0, 1, 2, 3
CLS_NONE, CLS_DIFFUSE, CLS_GLOSSY = 0, 1, 2
MODES = {"independent": INDEPENDENT, "morton_sort": MORTON_SORT,
         "direction_reuse": DIRECTION_REUSE, "world_reuse": WORLD_REUSE}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, IEEE float, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class _Params(C.Structure):
    _fields_ = [("spp", C.c_uint32), ("max_bounces", C.c_uint32), ("mode", C.c_uint32),
                ("tile_w", C.c_uint32), ("tile_h", C.c_uint32), ("k", C.c_uint32),
                ("interleave", C.c_uint32), ("frame_base", C.c_uint32), ("reuse_depth", C.c_uint32),
                ("opts", C.c_uint32), ("seed", C.c_uint64), ("diffuse_roughness", C.c_float)]


class _Outputs(C.Structure):
    _fields_ = [("accum", C.c_void_p), ("taint", C.c_void_p), ("dbg_prim", C.c_void_p),
                ("dbg_cat", C.c_void_p), ("dbg_cls", C.c_void_p), ("dbg_flags", C.c_void_p),
                ("dbg_local", C.c_void_p), ("dbg_world", C.c_void_p), ("counters", C.c_void_p),
                ("dbg_ray", C.c_void_p), ("dbg_t", C.c_void_p), ("dbg_beta", C.c_void_p)]


class _ReplayIn(C.Structure):
    _fields_ = [("ray", C.c_void_p), ("prim", C.c_void_p), ("t", C.c_void_p), ("beta", C.c_void_p)]


class _ReplayOut(C.Structure):
    _fields_ = [("dL", C.c_void_p), ("next_o", C.c_void_p), ("next_beta", C.c_void_p), ("next_pdf", C.c_void_p),
                ("next_alive", C.c_void_p), ("staint", C.c_void_p), ("cat", C.c_void_p), ("cls", C.c_void_p),
                ("flags", C.c_void_p), ("local", C.c_void_p), ("world", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, u32, i32 = C.c_void_p, C.c_uint32, C.c_int
        L.orc_philox4x32_10.argtypes = [u32, u32, vp, vp]
        L.orc_lcg_sequence.argtypes = [u32, u32, u32, u32, vp]
        L.orc_tile_sigma.argtypes = [u32, u32, u32, u32, C.c_uint64, i32, vp, vp]
        L.orc_sincos.argtypes = [C.c_float, vp, vp]
        L.orc_sample_cosine.argtypes = [C.c_float, C.c_float, vp]
        L.orc_sample_ggx.argtypes = [vp, C.c_float, vp, C.c_float, C.c_float, vp, vp]
        L.orc_sample_ggx.restype = i32
        L.orc_frame.argtypes = [vp, vp, vp]
        L.orc_sample_dielectric.argtypes = [vp, C.c_float, i32, C.c_float, vp]
        L.orc_sample_dielectric.restype = i32
        L.orc_scene_new.argtypes = [vp, u32, vp, vp, vp, u32, vp]
        L.orc_scene_new.restype = vp
        L.orc_scene_free.argtypes = [vp]
        L.orc_scene_nodes.argtypes = [vp]
        L.orc_scene_nodes.restype = u32
        L.orc_trace.argtypes = [vp, vp, vp, u32, i32, vp, vp, vp]
        L.orc_shadow.argtypes = [vp, vp, vp, u32, i32, vp, vp]
        L.orc_triangle_area.argtypes = [vp]
        L.orc_triangle_area.restype = C.c_double
        L.orc_scene_lights.argtypes = [vp, vp]
        L.orc_scene_lights.restype = u32
        L.orc_light_sample.argtypes = [vp, C.c_float, C.c_float, C.c_float, vp]
        L.orc_light_sample.restype = C.c_int32
        L.orc_eval_ggx.argtypes = [vp, vp, C.c_float, vp, vp]
        L.orc_pdf_ggx.argtypes = [vp, vp, C.c_float]
        L.orc_pdf_ggx.restype = C.c_double
        L.orc_render_tiles.argtypes = [vp, C.POINTER(_Camera), C.POINTER(_Params), u32, u32,
                                       C.POINTER(_Outputs)]
        L.orc_trace_bound.argtypes = [vp, vp, vp, u32, i32, vp, vp, vp, vp]
        L.orc_replay_step.argtypes = [vp, C.POINTER(_Camera), C.POINTER(_Params), u32, u32, u32, u32,
                                      C.POINTER(_ReplayIn), C.POINTER(_ReplayOut)]
        L.orc_camera_ray.argtypes = [C.POINTER(_Camera), u32, u32, C.c_float, C.c_float, vp]
        L.orc_spawn_point.argtypes = [vp, vp, C.c_double, vp, C.c_double, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox(key: int, ctr) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(key & 0xFFFFFFFF, (key >> 32) & 0xFFFFFFFF, _p(c), _p(out))
    return out


def lcg_sequence(m, a, c, x0) -> np.ndarray:
    out = np.zeros(m, dtype=np.uint32)
    lib().orc_lcg_sequence(m, a, c, x0, _p(out))
    return out


def tile_sigma(tile_w, tile_h, tile, frame, seed, lcg=True):
    out = np.zeros(tile_w * tile_h, dtype=np.uint32)
    abc = np.zeros(3, dtype=np.uint32)
    lib().orc_tile_sigma(tile_w, tile_h, tile, frame, seed, int(lcg), _p(out), _p(abc))
    return out, abc


def sincos(x: float):
    s = np.zeros(1, dtype=np.float32)
    c = np.zeros(1, dtype=np.float32)
    lib().orc_sincos(float(np.float32(x)), _p(s), _p(c))
    return s[0], c[0]


def sample_cosine(u1, u2):
    w = np.zeros(3, dtype=np.float32)
    lib().orc_sample_cosine(float(np.float32(u1)), float(np.float32(u2)), _p(w))
    return w


def sample_ggx(wo, alpha, f0, u1, u2):
    wo = np.ascontiguousarray(wo, dtype=np.float32)
    f0 = np.ascontiguousarray(f0, dtype=np.float32)
    wi = np.zeros(3, dtype=np.float32)
    wt = np.zeros(3, dtype=np.float32)
    ok = lib().orc_sample_ggx(_p(wo), float(np.float32(alpha)), _p(f0), float(np.float32(u1)),
                              float(np.float32(u2)), _p(wi), _p(wt))
    return bool(ok), wi, wt


def sample_dielectric(wo, eta, front, u):
    """-> (refracted?, wi float32[3]) of a smooth dielectric (IOR eta, entering if front)."""
    wo = np.ascontiguousarray(wo, dtype=np.float32)
    wi = np.zeros(3, dtype=np.float32)
    r = lib().orc_sample_dielectric(_p(wo), float(np.float32(eta)), int(bool(front)), float(np.float32(u)), _p(wi))
    return bool(r), wi


def frame(n):
    n = np.ascontiguousarray(n, dtype=np.float32)
    t = np.zeros(3, dtype=np.float32)
    b = np.zeros(3, dtype=np.float32)
    lib().orc_frame(_p(n), _p(t), _p(b))
    return t, b


class Scene:
    """Oracle copy of a scene (its own FP64 median-split BVH)."""

    def __init__(self, sc):
        self.src = sc
        self._arrays = (np.ascontiguousarray(sc.tri_xyz, dtype=np.float32),
                        np.ascontiguousarray(sc.tri_mat, dtype=np.uint32),
                        np.ascontiguousarray(sc.mat_type, dtype=np.uint32),
                        np.ascontiguousarray(sc.mat_params, dtype=np.float32),
                        np.ascontiguousarray(sc.env, dtype=np.float32))
        tx, tm, mt, mp, env = self._arrays
        self.h = lib().orc_scene_new(_p(tx), tx.shape[0], _p(tm), _p(mt), _p(mp), mt.shape[0], _p(env))

    @property
    def n_nodes(self):
        return lib().orc_scene_nodes(self.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_scene_free(self.h)
            self.h = None


def eval_ggx(wo, wi, alpha, f0):
    """GGX BSDF value f(wo, wi) (tangent frame) -> float64[3]."""
    wo = np.ascontiguousarray(wo, dtype=np.float32)
    wi = np.ascontiguousarray(wi, dtype=np.float32)
    f0 = np.ascontiguousarray(f0, dtype=np.float32)
    f = np.zeros(3, dtype=np.float64)
    lib().orc_eval_ggx(_p(wo), _p(wi), float(np.float32(alpha)), _p(f0), _p(f))
    return f


def pdf_ggx(wo, wi, alpha) -> float:
    """Solid-angle density of sample_ggx's direction wi."""
    wo = np.ascontiguousarray(wo, dtype=np.float32)
    wi = np.ascontiguousarray(wi, dtype=np.float32)
    return lib().orc_pdf_ggx(_p(wo), _p(wi), float(np.float32(alpha)))


def triangle_area(v9) -> float:
    v = np.ascontiguousarray(v9, dtype=np.float32).reshape(9)
    return lib().orc_triangle_area(_p(v))


def lights(scene) -> tuple:
    """(number of emitter triangles, total emitter area as float32)."""
    tot = np.zeros(1, dtype=np.float32)
    n = lib().orc_scene_lights(scene.h, _p(tot))
    return n, tot[0]


def light_sample(scene, u0, u1, u2):
    """-> (emitter's original triangle index, point float32[3])."""
    p = np.zeros(3, dtype=np.float32)
    t = lib().orc_light_sample(scene.h, float(np.float32(u0)), float(np.float32(u1)), float(np.float32(u2)), _p(p))
    return t, p


def shadow(scene, rays, skip=None, use_bvh=True):
    """Visibility of (n, 8) fp32 shadow rays (tmax in column 7) -> (occluded, fragile) uint8."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    n = rays.shape[0]
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int32)
    occ = np.zeros(n, dtype=np.uint8)
    fr = np.zeros(n, dtype=np.uint8)
    lib().orc_shadow(scene.h, _p(rays), _p(sk), n, int(use_bvh), _p(occ), _p(fr))
    return occ, fr


def trace(scene: Scene, rays, skip=None, use_bvh=True):
    """Closest hit of (n, 8) fp32 rays -> (prim int32, t float64, fragile uint8)."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    n = rays.shape[0]
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int32)
    prim = np.zeros(n, dtype=np.int32)
    t = np.zeros(n, dtype=np.float64)
    fr = np.zeros(n, dtype=np.uint8)
    lib().orc_trace(scene.h, _p(rays), _p(sk), n, int(use_bvh), _p(prim), _p(t), _p(fr))
    return prim, t, fr


def trace_bound(scene: Scene, rays, skip=None, use_bvh=True):
    """trace() plus the FP32 error scale of each winning hit's t (0 on a miss)."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    n = rays.shape[0]
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int32)
    prim = np.zeros(n, dtype=np.int32)
    t = np.zeros(n, dtype=np.float64)
    fr = np.zeros(n, dtype=np.uint8)
    terr = np.zeros(n, dtype=np.float64)
    lib().orc_trace_bound(scene.h, _p(rays), _p(sk), n, int(use_bvh), _p(prim), _p(t), _p(fr), _p(terr))
    return prim, t, fr, terr


def _camc(cam):
    return _Camera((C.c_float * 3)(*cam.pos), (C.c_float * 3)(*cam.look_at), (C.c_float * 3)(*cam.up),
                   cam.vfov_deg, cam.width, cam.height)


def camera_ray(cam, px, py, u, v):
    """Primary ray direction (float32[3]) through pixel (px, py) jittered by (u, v)."""
    d = np.zeros(3, dtype=np.float32)
    lib().orc_camera_ray(C.byref(_camc(cam)), int(px), int(py), float(np.float32(u)), float(np.float32(v)), _p(d))
    return d


def spawn_point(o, d, t, n, side=1.0):
    """Spawn point (float64[3]) of a ray leaving the surface hit at o + t d with normal n."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float32)
    n = np.ascontiguousarray(n, dtype=np.float32)
    out = np.zeros(3, dtype=np.float64)
    lib().orc_spawn_point(_p(o), _p(d), float(t), _p(n), float(side), _p(out))
    return out


def _params(spp, B, mode, tile, K, interleave, frame_base, reuse_depth, nee, hybrid_donor, nee_shared, seed,
            diffuse_roughness):
    W, H = tile
    return _Params(spp, B, MODES[mode] if isinstance(mode, str) else mode, W, H, K, int(interleave),
                   frame_base, reuse_depth, (1 if nee else 0) | (2 if hybrid_donor else 0) | (4 if nee_shared else 0),
                   seed, float(diffuse_roughness))


def replay_step(scene: Scene, cam, bounce, ray, prim, t, beta, *, max_bounces, mode="direction_reuse",
                tile=(8, 8), k=None, interleave=True, seed=0, frame=0, reuse_depth=0, nee=False,
                hybrid_donor=False, nee_shared=False, diffuse_roughness=0.0, tiles=None, threads=None):
    """Replay mode: recompute shading step ``bounce`` (1..B; B + 1 = the end of the last ray)
    of one frame from another renderer's captured inputs of trace bounce-1, per pixel:
    ``ray`` (npx, 8) float32, ``prim`` (npx,) int32 (-2 = not traced), ``t`` (npx,) float32,
    ``beta`` (npx, 4) float32.  Returns a dict of per-pixel arrays: dL, next_o, next_beta,
    next_pdf, next_alive, staint, cat, cls, flags, local, world."""
    W, H = tile
    K = W * H if k is None else k
    w, h = cam.width, cam.height
    npx = w * h
    ntiles = ((w + W - 1) // W) * ((h + H - 1) // H)
    t0, t1 = (0, ntiles) if tiles is None else tiles
    ray = np.ascontiguousarray(ray, dtype=np.float32).reshape(npx, 8)
    prim = np.ascontiguousarray(prim, dtype=np.int32).reshape(npx)
    t = np.ascontiguousarray(t, dtype=np.float32).reshape(npx)
    beta = np.ascontiguousarray(beta, dtype=np.float32).reshape(npx, 4)
    res = dict(dL=np.zeros((npx, 3)), next_o=np.full((npx, 3), np.nan), next_beta=np.full((npx, 3), np.nan, np.float32),
               next_pdf=np.full(npx, np.nan), next_alive=np.zeros(npx, np.uint8), staint=np.zeros(npx, np.uint8),
               cat=np.full(npx, 255, np.uint8), cls=np.zeros(npx, np.uint8), flags=np.zeros(npx, np.uint8),
               local=np.zeros((npx, 3), np.float32), world=np.zeros((npx, 3), np.float32))
    camc = _camc(cam)
    par = _params(1, max_bounces, mode, tile, K, interleave, frame, reuse_depth, nee, hybrid_donor, nee_shared,
                  seed, diffuse_roughness)
    rin = _ReplayIn(_p(ray), _p(prim), _p(t), _p(beta))
    rout = _ReplayOut(*[_p(res[key]) for key in ("dL", "next_o", "next_beta", "next_pdf", "next_alive", "staint",
                                                 "cat", "cls", "flags", "local", "world")])
    nthreads = threads or max(1, min(os.cpu_count() or 1, t1 - t0))
    bounds = np.linspace(t0, t1, nthreads + 1).astype(int)

    def work(i):
        lib().orc_replay_step(scene.h, C.byref(camc), C.byref(par), frame, bounce, int(bounds[i]),
                              int(bounds[i + 1]), C.byref(rin), C.byref(rout))

    ths = [threading.Thread(target=work, args=(i,)) for i in range(nthreads) if bounds[i] < bounds[i + 1]]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return res


def render(scene: Scene, cam, *, spp=1, max_bounces=1, mode="direction_reuse", tile=(8, 8), k=None,
           interleave=True, seed=0, frame_base=0, reuse_depth=0, debug=False, threads=None,
           tiles=None, accum=None, nee=False, hybrid_donor=False, nee_shared=False, diffuse_roughness=0.0):
    """Run the oracle path tracer.  Returns a dict with ``rgb`` (mean radiance, float64 h x w x 3),
    ``taint`` (h x w uint8), ``counters`` and, with debug=True (spp 1), per-bounce arrays
    (debug="replay" adds the replay capture: ray, t, beta of every trace).
    ``tiles`` = (begin, end) restricts the work to a tile range (other pixels stay 0).
    ``accum`` (npx x 3 float64) continues an earlier accumulation in place (progressive
    rendering resumed at ``frame_base``).  ``nee`` adds next-event estimation (one light
    sample and shadow ray per non-specular shading point).  ``hybrid_donor`` makes the diffuse
    members of hybrid groups reuse the first diffuse member's own sample instead of the
    average glossy direction (an unbiased option).  ``nee_shared`` (with ``nee``) makes the
    members of a group join one light point.  ``diffuse_roughness`` > 0 puts GGX points of at
    least that roughness in the diffuse class where directions are reused (cosine samples,
    weight pi f)."""
    W, H = tile
    K = W * H if k is None else k
    w, h = cam.width, cam.height
    npx = w * h
    B = max_bounces
    ntiles = ((w + W - 1) // W) * ((h + H - 1) // H)
    t0, t1 = (0, ntiles) if tiles is None else tiles
    if accum is None:
        accum = np.zeros((npx, 3), dtype=np.float64)
    assert accum.shape == (npx, 3) and accum.dtype == np.float64 and accum.flags.c_contiguous
    taint = np.zeros(npx, dtype=np.uint8)
    dbg = {}
    if debug:
        dbg = dict(prim=np.full((B + 1, npx), -2, dtype=np.int32), cat=np.full((B, npx), 255, np.uint8),
                   cls=np.zeros((B, npx), np.uint8), flags=np.zeros((B, npx), np.uint8),
                   local=np.zeros((B, npx, 3), np.float32), world=np.zeros((B, npx, 3), np.float32))
        if debug == "replay":
            dbg.update(ray=np.zeros((B + 1, npx, 8), np.float32), t=np.full((B + 1, npx), np.nan, np.float32),
                       beta=np.zeros((B + 1, npx, 4), np.float32))
    camc = _Camera((C.c_float * 3)(*cam.pos), (C.c_float * 3)(*cam.look_at), (C.c_float * 3)(*cam.up),
                   cam.vfov_deg, w, h)
    par = _Params(spp, B, MODES[mode] if isinstance(mode, str) else mode, W, H, K, int(interleave),
                  frame_base, reuse_depth, (1 if nee else 0) | (2 if hybrid_donor else 0) | (4 if nee_shared else 0),
                  seed, float(diffuse_roughness))
    nthreads = threads or max(1, min(os.cpu_count() or 1, t1 - t0))
    bounds = np.linspace(t0, t1, nthreads + 1).astype(int)
    counters = np.zeros((nthreads, 5), dtype=np.uint64)

    def work(i):
        o = _Outputs(_p(accum), _p(taint), _p(dbg.get("prim")), _p(dbg.get("cat")), _p(dbg.get("cls")),
                     _p(dbg.get("flags")), _p(dbg.get("local")), _p(dbg.get("world")), _p(counters[i]),
                     _p(dbg.get("ray")), _p(dbg.get("t")), _p(dbg.get("beta")))
        lib().orc_render_tiles(scene.h, C.byref(camc), C.byref(par), int(bounds[i]), int(bounds[i + 1]),
                               C.byref(o))

    ths = [threading.Thread(target=work, args=(i,)) for i in range(nthreads) if bounds[i] < bounds[i + 1]]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    res = dict(rgb=(accum / spp).reshape(h, w, 3), accum=accum, taint=taint.reshape(h, w),
               counters=counters.sum(axis=0), threads=len(ths))
    for key, v in dbg.items():
        res["dbg_" + key] = v
    return res
