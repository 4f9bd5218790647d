"""CPU pins of the oracle's replay mode, camera, spawn point and t error bound.

Replay mode recomputes one shading step (Sec. 3.2: shade, classify, reuse, spawn) from a
renderer's captured inputs of the previous trace.  Replaying the oracle's own capture must
give back exactly what its render computed, step by step: the same categories, classes and
exit directions, the same spawned rays and throughputs, and the same radiance."""
import math

import numpy as np
import pytest

from paper_2310_07182_gb300 import scenes
from replay_util import T_ERR_K, spawn_tolerance


def _replay_all(orc, O, cam, ref, B, **kw):
    """Replay every step of a captured spp-1 render; returns the per-step outputs."""
    steps = []
    for b in range(1, B + 2):
        steps.append(orc.replay_step(O, cam, b, ref["dbg_ray"][b - 1], ref["dbg_prim"][b - 1],
                                     ref["dbg_t"][b - 1], ref["dbg_beta"][b - 1], max_bounces=B, **kw))
    return steps


def _check_self_replay(orc, sc, B, nee=False, **kw):
    O = orc.Scene(sc)
    cam = sc.camera
    ref = orc.render(O, cam, spp=1, max_bounces=B, debug="replay", nee=nee, **kw)
    kw.pop("frame_base", None)
    steps = _replay_all(orc, O, cam, ref, B, frame=0, nee=nee, **kw)
    npx = cam.width * cam.height
    for b in range(1, B + 1):
        st = steps[b - 1]
        assert np.array_equal(st["cat"], ref["dbg_cat"][b - 1])
        assert np.array_equal(st["cls"], ref["dbg_cls"][b - 1])
        assert np.array_equal(st["flags"] & 3, ref["dbg_flags"][b - 1] & 3)
        assert np.array_equal(st["local"].view(np.uint32), ref["dbg_local"][b - 1].view(np.uint32))
        assert np.array_equal(st["world"].view(np.uint32), ref["dbg_world"][b - 1].view(np.uint32))
        traced = ref["dbg_prim"][b] != -2
        assert np.array_equal(st["next_alive"].astype(bool), traced)
        # the spawned ray is the ray of the next trace: direction and throughput bit for bit,
        # origin up to the capture's rounding to float
        ray = ref["dbg_ray"][b]
        assert np.array_equal(st["world"][traced].view(np.uint32), ray[traced, 4:7].view(np.uint32))
        assert np.array_equal(st["next_beta"][traced].view(np.uint32),
                              ref["dbg_beta"][b][traced, :3].view(np.uint32))
        prev = ref["dbg_ray"][b - 1][traced]
        tol = spawn_tolerance(prev[:, :3], prev[:, 4:7], ref["dbg_t"][b - 1][traced], ray[traced, :3])
        assert (np.abs(st["next_o"][traced] - ray[traced, :3]) <= tol).all()
        assert np.array_equal(st["next_pdf"][traced].astype(np.float32), ref["dbg_beta"][b][traced, 3])
    L = sum(st["dL"] for st in steps).reshape(cam.height, cam.width, 3)
    if nee:
        # light samples leave from spawn points rebuilt from the float-rounded t
        ok = sum(st["staint"] for st in steps).reshape(cam.height, cam.width) == 0
        assert ok.mean() > 0.99
        # the parity criterion (relative, with an absolute floor below 1e-2), ten times tighter
        assert (np.abs(L[ok] - ref["rgb"][ok]) <= 1e-5 * np.maximum(np.abs(ref["rgb"][ok]), 1e-2)).all()
    else:
        np.testing.assert_allclose(L, ref["rgb"], rtol=1e-12, atol=0)
    assert npx == L.shape[0] * L.shape[1]
    return ref, steps


@pytest.mark.parametrize("mode,k,interleave", [("direction_reuse", 4, True), ("direction_reuse", 16, False),
                                               ("independent", 16, True), ("world_reuse", 8, True)])
def test_replay_of_own_capture_reproduces_the_render(orc, mode, k, interleave):
    sc = scenes.tiny(material_mix="mixed", n_soup=1500, width=48, height=40)
    _check_self_replay(orc, sc, 3, mode=mode, tile=(4, 4), k=k, interleave=interleave, seed=7)


def test_replay_block_groups_and_hybrid_donor(orc):
    sc = scenes.tiny(material_mix="mixed", n_soup=1500, width=48, height=40)
    _check_self_replay(orc, sc, 2, mode="direction_reuse", tile=(8, 8), k=64, seed=3, hybrid_donor=True)
    _check_self_replay(orc, sc, 2, mode="direction_reuse", tile=(8, 8), k=8, seed=3, diffuse_roughness=0.3)


def test_replay_with_next_event_estimation(orc):
    sc = scenes.interior(width=40, height=32)
    _check_self_replay(orc, sc, 3, nee=True, mode="direction_reuse", tile=(8, 8), k=8, seed=5)
    _check_self_replay(orc, sc, 3, nee=True, nee_shared=True, mode="direction_reuse", tile=(8, 8), k=8, seed=5)


def test_replay_with_transmission(orc):
    sc = scenes.tiny(material_mix="transmissive", n_soup=1500, width=40, height=32)
    _check_self_replay(orc, sc, 4, mode="direction_reuse", tile=(4, 4), k=8, seed=2)


def test_replay_detects_a_changed_input(orc):
    """The replay works on its inputs, not on a render of its own: a planted wrong hit for
    one pixel changes that pixel's shading outputs."""
    sc = scenes.tiny(material_mix="mixed", n_soup=1500, width=32, height=32)
    O = orc.Scene(sc)
    cam = sc.camera
    ref = orc.render(O, cam, spp=1, max_bounces=1, debug="replay", tile=(4, 4), k=1, seed=1)
    prim = ref["dbg_prim"][0].copy()
    hit = np.flatnonzero(prim >= 0)
    pix = int(hit[len(hit) // 2])
    prim[pix] = sc.tri_xyz.shape[0] - 1 if prim[pix] != sc.tri_xyz.shape[0] - 1 else 0  # the other ground triangle or a soup triangle
    st = orc.replay_step(O, cam, 1, ref["dbg_ray"][0], prim, ref["dbg_t"][0], ref["dbg_beta"][0], max_bounces=1,
                         tile=(4, 4), k=1, seed=1)
    changed = np.flatnonzero((st["world"] != ref["dbg_world"][0]).any(axis=1))
    assert pix in changed.tolist() and len(changed) == 1


# ------------------------------------------------------------------------------------
# Camera (the pinhole of the primary rays, Sec. 3.1 "one path per pixel"): closed forms.

def _angle(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return math.acos(max(-1.0, min(1.0, float(a @ b / np.linalg.norm(a) / np.linalg.norm(b)))))


@pytest.mark.parametrize("w,h,vfov", [(64, 64, 60.0), (1920, 1080, 50.0), (53, 29, 55.0), (32, 96, 90.0)])
def test_camera_closed_forms(orc, w, h, vfov):
    pos, look = (0.5, 2.0, -3.0), (1.5, 1.0, 4.0)
    cam = scenes.Camera(pos, look, (0.0, 1.0, 0.0), vfov, w, h)
    fwd = np.subtract(look, pos).astype(np.float64)
    fwd /= np.linalg.norm(fwd)
    # the image centre looks at look_at: (px + u) / w = (py + v) / h = 1/2
    c = orc.camera_ray(cam, w // 2, h // 2, 0.5 * (w % 2), 0.5 * (h % 2))
    assert _angle(c, fwd) < 4e-7
    top = orc.camera_ray(cam, w // 2, 0, 0.5 * (w % 2), 0.0)
    bottom = orc.camera_ray(cam, w // 2, h, 0.5 * (w % 2), 0.0)
    left = orc.camera_ray(cam, 0, h // 2, 0.0, 0.5 * (h % 2))
    right = orc.camera_ray(cam, w, h // 2, 0.0, 0.5 * (h % 2))
    # vfov is the vertical field of view; the horizontal one follows from the aspect ratio
    assert abs(_angle(top, bottom) - math.radians(vfov)) < 2e-6
    hfov = 2.0 * math.atan(w / h * math.tan(math.radians(vfov) / 2.0))
    assert abs(_angle(left, right) - hfov) < 2e-6
    # row 0 is the top of the image; column 0 is its left: the camera frame (right, up, -fwd)
    # is right-handed, with right = fwd x up
    up_w = np.array([0.0, 1.0, 0.0])
    right_w = np.cross(fwd, up_w)
    assert top @ up_w > c @ up_w > bottom @ up_w
    assert left @ right_w < 0 < right @ right_w
    # every primary direction is unit length in float
    for d in (c, top, bottom, left, right):
        assert abs(float(np.linalg.norm(d.astype(np.float64))) - 1.0) < 3e-7


def test_camera_jitter_moves_within_the_pixel(orc):
    cam = scenes.Camera((0, 0, -3), (0, 0, 0), (0, 1, 0), 60.0, 16, 16)
    a = orc.camera_ray(cam, 5, 7, 0.0, 0.0)
    b = orc.camera_ray(cam, 5, 7, 0.999, 0.999)
    nxt = orc.camera_ray(cam, 6, 8, 0.0, 0.0)
    # (px + u) is continuous: the far corner of pixel (5, 7) is the near corner of (6, 8)
    assert _angle(b, nxt) < 2e-3 * _angle(a, nxt)  # a gap of 0.001 of the pixel diagonal


# ------------------------------------------------------------------------------------
# Spawn point: p = o + t d, offset by 2^-18 max(1, |p|_inf) along +-n.

def test_spawn_point_closed_forms(orc):
    z = orc.spawn_point([0, 0, 0], [0, 0, 1], 2.0, [0, 0, -1], 1.0)
    assert z.tolist() == [0.0, 0.0, 2.0 - 2.0 ** -17]
    z = orc.spawn_point([0, 0, 0], [0, 0, 1], 2.0, [0, 0, -1], -1.0)  # transmitted: through the surface
    assert z.tolist() == [0.0, 0.0, 2.0 + 2.0 ** -17]
    z = orc.spawn_point([0.25, 0, 0], [0, 1, 0], 0.5, [0, -1, 0], 1.0)  # |p| < 1: eps = 2^-18
    assert z.tolist() == [0.25, 0.5 - 2.0 ** -18, 0.0]
    z = orc.spawn_point([-8, 1, 3], [0, 0, 1], 0.0, [1, 0, 0], 1.0)  # |p|_inf = 8
    assert z.tolist() == [-8.0 + 2.0 ** -15, 1.0, 3.0]


def test_spawn_point_leaves_the_plane_on_the_requested_side(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        n = n.astype(np.float32)
        o = rng.uniform(-50, 50, size=3)
        d = rng.normal(size=3).astype(np.float32)
        t = float(rng.uniform(0.1, 20))
        p = o + t * d.astype(np.float64)
        eps = 2.0 ** -18 * max(1.0, float(np.abs(p).max()))
        for side in (1.0, -1.0):
            q = orc.spawn_point(o, d, t, n, side)
            h = float((q - p) @ n.astype(np.float64))
            assert abs(h - side * eps) <= 1e-9 * eps + 1e-12 * np.abs(p).max()


# ------------------------------------------------------------------------------------
# t error bound: terr must bound the error of an FP32 intersector's t.

def _mt_f32(o, d, v0, v1, v2):
    """Moller-Trumbore in float32, each operation rounded (numpy scalar float32)."""
    f = np.float32
    e1 = (v1 - v0).astype(f)
    e2 = (v2 - v0).astype(f)
    pv = np.cross(d, e2).astype(f)
    det = f(f(e1[0] * pv[0] + e1[1] * pv[1]) + e1[2] * pv[2])
    tv = (o - v0).astype(f)
    qv = np.cross(tv, e1).astype(f)
    num = f(f(e2[0] * qv[0] + e2[1] * qv[1]) + e2[2] * qv[2])
    return f(num / det)


def test_t_error_bound_covers_an_fp32_intersector(orc):
    """terr is 4 rounding units of the coordinate magnitude over the ray's obliquity to the
    triangle; an FP32 t passes through about 16 roundings of that magnitude (differences,
    cross and dot products, one division), so T_ERR_K = 4 units of terr bound it."""
    rng = np.random.default_rng(11)
    tris, rays = [], []
    for i in range(400):
        c = rng.uniform(-200, 200, size=3)
        v = (c + rng.normal(scale=rng.uniform(0.05, 5.0), size=(3, 3))).astype(np.float32)
        o = (c + rng.normal(scale=50, size=3)).astype(np.float32)
        target = (v[0] * 0.3 + v[1] * 0.3 + v[2] * 0.4).astype(np.float64)
        d = (target - o.astype(np.float64)).astype(np.float32)
        d /= np.float32(np.linalg.norm(d.astype(np.float64)) * rng.uniform(0.2, 3.0))
        tris.append(v.reshape(9))
        rays.append(np.r_[o, 0.0, d, np.inf].astype(np.float32))
    sc = scenes.Scene(name="tbound", tri_xyz=np.array(tris, np.float32), tri_mat=np.zeros(len(tris), np.uint32),
                      mat_type=np.zeros(1, np.uint32), mat_params=np.array([[0.5, 0.5, 0.5, 0, 0, 0, 0]], np.float32),
                      env=np.ones(3, np.float32), camera=None)
    O = orc.Scene(sc)
    checked = 0
    for i, r in enumerate(rays):
        prim, t, fr, terr = orc.trace_bound(O, r[None], None)
        if prim[0] != i or fr[0] & 1:
            continue  # another triangle is closer, or the decision is too close to call
        t32 = _mt_f32(r[:3], r[4:7], *np.array(tris[i], np.float32).reshape(3, 3))
        assert abs(float(t32) - t[0]) <= T_ERR_K * terr[0], (i, float(t32), t[0], terr[0])
        checked += 1
    assert checked > 300
