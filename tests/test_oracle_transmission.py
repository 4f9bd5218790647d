"""Pins of the oracle's transmission materials (the paper's future work, Sec. 6): the smooth
dielectric against Fresnel's and Snell's closed forms and a glass slab, the Lambertian
transmitter against a closed emitting box, and the lower-hemisphere reuse rule (a shared
tangent-space direction mirrored into each member's own lobe) against its invariants and
against independent sampling."""
import math

import numpy as np
import pytest

from paper_2310_07182_gb300 import scenes


def _fresnel(eta_i, eta_t, ci):
    s2 = (eta_i / eta_t) ** 2 * (1 - ci * ci)
    if s2 >= 1:
        return 1.0
    ct = math.sqrt(1 - s2)
    rs = (eta_i * ci - eta_t * ct) / (eta_i * ci + eta_t * ct)
    rp = (eta_t * ci - eta_i * ct) / (eta_t * ci + eta_i * ct)
    return 0.5 * (rs * rs + rp * rp)


@pytest.mark.parametrize("eta", [1.33, 1.5, 2.4])
def test_dielectric_normal_incidence_reflectance(orc, eta):
    N = 20000
    refl = sum(not orc.sample_dielectric([0, 0, 1], eta, True, (i + 0.5) / N)[0] for i in range(N))
    assert abs(refl / N - ((eta - 1) / (eta + 1)) ** 2) < 2.0 / N


def test_dielectric_snell_fresnel_and_total_internal_reflection(orc):
    eta = 1.5
    for th in np.linspace(0.05, 1.5, 12):
        wo = np.float32([math.sin(th) * 0.6, math.sin(th) * 0.8, math.cos(th)])
        for front in (True, False):
            eta_i, eta_t = (1.0, eta) if front else (eta, 1.0)
            F = _fresnel(eta_i, eta_t, float(wo[2]))
            N = 4000
            n_refl = 0
            for i in range(N):
                refr, wi = orc.sample_dielectric(wo, eta, front, (i + 0.5) / N)
                if not refr:
                    n_refl += 1
                    assert np.allclose(wi, [-wo[0], -wo[1], wo[2]])
                else:
                    # Snell: sin_t = (eta_i / eta_t) sin_i, opposite tangential direction,
                    # lower hemisphere, unit length
                    si = math.hypot(wo[0], wo[1])
                    st = math.hypot(wi[0], wi[1])
                    assert st == pytest.approx(eta_i / eta_t * si, rel=1e-5, abs=1e-7)
                    assert wi[2] < 0 and np.linalg.norm(wi) == pytest.approx(1.0, abs=1e-6)
                    assert np.dot(wi[:2], wo[:2]) <= 0
            assert abs(n_refl / N - F) < 2.0 / N, (th, front, n_refl / N, F)
            if not front and math.sin(th) > 1 / eta:
                assert n_refl == N  # total internal reflection


def _slab(eta=1.5, width=32, height=32):
    """A glass box 4 x 4 x 0.5 (outward faces) seen head-on, an emitter wall behind it."""
    box = scenes._box_room((-2.0, -2.0, -0.25), (2.0, 2.0, 0.25))
    # orient every face outward (cross(e1, e2) away from the centre)
    t = box.reshape(-1, 3, 3)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    flip = (n * t.mean(axis=1)).sum(axis=1) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    wall = np.array([[-9, -9, 3, 9, -9, 3, 9, 9, 3], [-9, -9, 3, 9, 9, 3, -9, 9, 3]], np.float64)
    tris = np.concatenate([t.reshape(-1, 9), wall])
    mat = np.array([0] * 12 + [1, 1])
    params = np.zeros((2, 7))
    params[0, 0:4] = (1.0, 1.0, 1.0, eta)
    params[1, 4:7] = 1.0
    cam = scenes.Camera((0.3, -0.2, -3.0), (0.3, -0.2, 0.0), (0.0, 1.0, 0.0), 40.0, width, height)
    return scenes._finish("slab", tris, mat, [scenes.MAT_DIELECTRIC, scenes.MAT_EMITTER], params, (0, 0, 0), cam)


def test_glass_slab_exit_direction_equals_entry_direction(orc):
    """Through a parallel glass slab a ray leaves parallel to the way it came in.  The entry
    directions come from the same slab with IOR 1 (Fresnel 0, no bending: the bounce-1
    direction is the camera ray); at IOR 1.5 the bounce-2 (exit) direction must equal it,
    and inside the slab sin_t = sin_i / 1.5."""
    kw = dict(spp=1, max_bounces=2, mode="independent", tile=(8, 8), seed=3, debug=True)
    sc1 = _slab(eta=1.0)
    r1 = orc.render(orc.Scene(sc1), sc1.camera, **kw)
    cam_dir = r1["dbg_world"][0].reshape(-1, 3)
    sc = _slab()
    r = orc.render(orc.Scene(sc), sc.camera, **kw)
    w1 = r["dbg_world"][0].reshape(-1, 3)
    w2 = r["dbg_world"][1].reshape(-1, 3)
    through = (w1[:, 2] > 0) & (w2[:, 2] > 0)          # refracted in and out
    assert through.mean() > 0.8
    assert np.allclose(w2[through], cam_dir[through], atol=2e-6)
    si = np.hypot(cam_dir[through, 0], cam_dir[through, 1])
    st = np.hypot(w1[through, 0], w1[through, 1])
    assert np.allclose(st, si / 1.5, rtol=1e-5, atol=1e-7)
    # the ray is not bent at IOR 1, and the exit rays reach the emitter wall
    assert (r1["dbg_world"][1].reshape(-1, 3)[:, 2] > 0).all()
    assert (r["rgb"].reshape(-1, 3)[through] == 1.0).all()


def test_translucent_floor_transmits_into_the_emitting_box(orc):
    """Seen from below, a translucent floor sends every transmitted ray into the box whose
    five other walls emit: the pixel is exactly albedo * le (a reflected ray would see the
    black environment); with next-event estimation the mean is the same."""
    alb = np.float32([0.6, 0.5, 0.4]).astype(np.float64)
    sc = scenes.emitter_box(floor=scenes.MAT_TRANSLUCENT, floor_params=(0.6, 0.5, 0.4, 0.0), width=16, height=16)
    sc.camera = scenes.Camera((0.1, -3.0, 0.2), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0), 30.0, 16, 16)
    S = orc.Scene(sc)
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="independent", tile=(8, 8), seed=2, debug=True)
    floor = np.isin(r["dbg_prim"][0], [8, 9]).reshape(16, 16)
    assert floor.mean() > 0.5
    assert np.array_equal(r["rgb"][floor], np.broadcast_to(alb, (floor.sum(), 3)))
    assert (r["dbg_cls"][0][floor.ravel()] == 3).all()
    assert (r["dbg_local"][0].reshape(-1, 3)[floor.ravel(), 2] < 0).all()
    nee = orc.render(S, sc.camera, spp=256, max_bounces=1, mode="independent", tile=(8, 8), seed=2, nee=True)
    v = nee["rgb"][floor]
    se = v.std(axis=0) / math.sqrt(v.shape[0])
    assert (np.abs(v.mean(axis=0) - alb) < 4 * se + 1e-9).all() and nee["counters"][3] > 0


def test_lower_hemisphere_reuse_shares_the_direction_mirrored(orc):
    """A plane of Lambert and translucent strips: every group is diffuse-class, and all its
    members take the donor's tangent-space direction with z = +|z| (Lambert) or -|z|
    (translucent)."""
    sc = scenes.split_plane(width=32, height=32, left=scenes.MAT_LAMBERT, right=scenes.MAT_TRANSLUCENT, n_strips=4)
    S = orc.Scene(sc)
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="direction_reuse", tile=(8, 8), k=16, seed=5, debug=True)
    cls = r["dbg_cls"][0]
    loc = r["dbg_local"][0].reshape(-1, 3)
    alive = cls > 0
    assert set(np.unique(cls[alive])) == {1, 3}
    assert (r["dbg_cat"][0][alive] == 1).all()
    assert (loc[cls == 1, 2] > 0).all() and (loc[cls == 3, 2] < 0).all()
    # group by the shared |direction|: within a group the (x, y, |z|) triple is one value
    key = np.round(np.column_stack([loc[:, 0], loc[:, 1], np.abs(loc[:, 2])]), 7)[alive]
    n_groups = len({tuple(k) for k in key})
    assert n_groups <= alive.sum() // 16 + 8
    mixed = 0
    for k in {tuple(k) for k in key}:
        members = cls[alive][(key == k).all(axis=1)]
        mixed += len(set(members)) > 1
    assert mixed > 0  # groups straddling a Lambert/translucent edge share one direction


def test_lower_hemisphere_reuse_is_unbiased(orc):
    sc = scenes.split_plane(width=16, height=16, left=scenes.MAT_LAMBERT, right=scenes.MAT_TRANSLUCENT, n_strips=4)
    S = orc.Scene(sc)
    means = {"independent": [], "direction_reuse": []}
    for f in range(40):
        for mode in means:
            r = orc.render(S, sc.camera, spp=1, max_bounces=2, mode=mode, tile=(4, 4), k=16, seed=9, frame_base=f)
            means[mode].append(r["rgb"].mean())
    a, b = np.array(means["independent"]), np.array(means["direction_reuse"])
    se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 5 * se + 1e-12


def test_transmissive_mix_renders_in_every_mode(orc):
    sc = scenes.tiny(material_mix="transmissive")
    S = orc.Scene(sc)
    for mode in ("independent", "direction_reuse", "morton_sort", "world_reuse"):
        r = orc.render(S, sc.camera, spp=2, max_bounces=3, mode=mode, tile=(4, 4), k=8, seed=4, nee=True)
        assert np.isfinite(r["rgb"]).all() and r["rgb"].mean() > 0.05
