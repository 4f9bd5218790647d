"""Pins of the oracle's next-event estimation (light sampling, GGX evaluation, shadow rays,
the estimator) against closed forms, brute force and plain path tracing."""
import numpy as np
import pytest

from paper_2310_07182_gb300 import scenes


def test_triangle_area_closed_forms(orc):
    assert orc.triangle_area([0, 0, 0, 3, 0, 0, 0, 4, 0]) == 6.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.normal(size=(3, 3)).astype(np.float32).astype(np.float64)
        a, b, c = (np.linalg.norm(v[i] - v[(i + 1) % 3]) for i in range(3))
        s = (a + b + c) / 2
        heron = np.sqrt(s * (s - a) * (s - b) * (s - c))
        assert orc.triangle_area(v) == pytest.approx(heron, rel=1e-9)


def _three_lights():
    """Three emitter triangles of areas 1, 2 and 5 among Lambert triangles."""
    tris = np.array([[0, 0, 0, 2, 0, 0, 0, 1, 0],        # emitter, area 1
                     [5, 5, 5, 6, 5, 5, 5, 6, 5],        # Lambert
                     [0, 0, 3, 2, 0, 3, 0, 2, 3],        # emitter, area 2
                     [0, 0, 6, 5, 0, 6, 0, 2, 6],        # emitter, area 5
                     [9, 9, 9, 9, 10, 9, 9, 9, 10]], np.float64)
    mat = np.array([1, 0, 1, 1, 0])
    params = np.zeros((2, 7))
    params[0, 0:3] = 0.5
    params[1, 4:7] = 3.0
    return scenes._finish("lights", tris, mat, [scenes.MAT_LAMBERT, scenes.MAT_EMITTER], params, (0, 0, 0), None)


def test_light_choice_proportional_to_area_and_points_uniform(orc):
    sc = _three_lights()
    S = orc.Scene(sc)
    n, total = orc.lights(S)
    assert n == 3 and total == np.float32(8.0)
    N = 4000
    counts = {0: 0, 2: 0, 3: 0}
    for i in range(N):
        t, _ = orc.light_sample(S, (i + 0.5) / N, 0.3, 0.6)
        counts[t] += 1
    assert abs(counts[0] / N - 1 / 8) < 2 / N
    assert abs(counts[2] / N - 2 / 8) < 2 / N
    assert abs(counts[3] / N - 5 / 8) < 2 / N
    # points: inside the chosen triangle, and their mean over a fine (u1, u2) grid is the centroid
    G = 64
    v = sc.tri_xyz[3].astype(np.float64).reshape(3, 3)
    pts = []
    for a in range(G):
        for b in range(G):
            t, p = orc.light_sample(S, 0.9, (a + 0.5) / G, (b + 0.5) / G)
            assert t == 3
            pts.append(p)
    pts = np.array(pts, np.float64)
    M = np.stack([v[1] - v[0], v[2] - v[0]], axis=1)[:2]   # the triangle lies in z = 6
    bc = np.linalg.solve(M, (pts[:, :2] - v[0, :2]).T).T
    assert (bc >= -1e-6).all() and (bc.sum(axis=1) <= 1 + 1e-6).all()
    assert np.allclose(pts[:, 2], 6.0)
    assert np.allclose(pts.mean(axis=0), v.mean(axis=0), atol=2e-3)


def test_no_emitter_no_light(orc):
    S = orc.Scene(scenes.tiny())
    assert orc.lights(S)[0] == 0
    assert orc.light_sample(S, 0.5, 0.5, 0.5)[0] == -1


def test_ggx_eval_normal_incidence_and_reciprocity(orc):
    for alpha in (0.1, 0.3, 0.7):
        f = orc.eval_ggx([0, 0, 1], [0, 0, 1], alpha, [0.2, 0.5, 1.0])
        # h = n: D = 1 / (pi alpha^2), G1 = 1, F = F0 -> f = F0 / (4 pi alpha^2)
        want = np.float32([0.2, 0.5, 1.0]).astype(np.float64) / (4 * np.pi * np.float32(alpha) ** 2)
        assert np.allclose(f, want, rtol=1e-6)
    rng = np.random.default_rng(3)
    for _ in range(200):
        a, b = rng.normal(size=(2, 3))
        a[2], b[2] = abs(a[2]), abs(b[2])
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        f1 = orc.eval_ggx(a, b, 0.35, [0.9, 0.5, 0.1])
        f2 = orc.eval_ggx(b, a, 0.35, [0.9, 0.5, 0.1])
        assert np.allclose(f1, f2, rtol=1e-5)
    assert (orc.eval_ggx([0, 0.6, 0.8], [0, 0.6, -0.8], 0.3, [1, 1, 1]) == 0).all()


@pytest.mark.parametrize("alpha", [0.15, 0.4])
def test_ggx_eval_integrates_to_the_sampler_mean_weight(orc, alpha):
    """int f cos dwi by quadrature over the hemisphere equals the mean importance weight of
    orc_sample_ggx over a stratified (u1, u2) grid: both are the directional albedo."""
    f0 = [0.9, 0.6, 0.3]
    wo = np.float32([np.sin(0.6), 0.0, np.cos(0.6)])
    G = 200
    wsum = np.zeros(3)
    for a in range(G):
        for b in range(G):
            ok, wi, wt = orc.sample_ggx(wo, alpha, f0, (a + 0.5) / G, (b + 0.5) / G)
            if ok:
                wsum += wt
    sampled = wsum / G ** 2
    # quadrature in (cos theta, phi), denser near the specular lobe
    nt, nphi = 400, 400
    mu = (np.arange(nt) + 0.5) / nt
    phi = (np.arange(nphi) + 0.5) / nphi * 2 * np.pi
    quad = np.zeros(3)
    for m in mu:
        st = np.sqrt(1 - m * m)
        for ph in phi:
            wi = [st * np.cos(ph), st * np.sin(ph), m]
            quad += orc.eval_ggx(wo, wi, alpha, f0) * m
    quad *= (1.0 / nt) * (2 * np.pi / nphi)
    assert np.allclose(quad, sampled, rtol=0.03), (quad, sampled)


def test_shadow_rays_match_brute_force(orc):
    sc = scenes.tiny(seed=5, n_soup=3000)
    S = orc.Scene(sc)
    rng = np.random.default_rng(8)
    n = 3000
    o = rng.uniform(-1.2, 1.2, size=(n, 3))
    q = rng.uniform(-1.2, 1.2, size=(n, 3))
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = q - o
    rays[:, 7] = 1.0 - 2.0 ** -10
    occ, fr = orc.shadow(S, rays)
    occ_b, fr_b = orc.shadow(S, rays, use_bvh=False)
    assert (fr == fr_b).all() and (occ == occ_b).all()
    assert 0.2 < occ.mean() < 0.95 and fr.mean() < 1e-3
    # against the closest hit: occluded iff the closest hit lies before tmax
    prim, t, cfr = orc.trace(S, rays)
    clean = (fr == 0) & ((cfr & 1) == 0)
    assert ((prim[clean] >= 0) & (t[clean] < rays[clean, 7])).tolist() == occ[clean].astype(bool).tolist()


def test_shadow_ray_hand_cases(orc):
    tris = np.array([[-1, -1, 2, 1, -1, 2, 0, 1, 2]], np.float64)
    sc = scenes._finish("one", tris, [0], [scenes.MAT_LAMBERT], np.zeros((1, 7)), (0, 0, 0), None)
    S = orc.Scene(sc)
    rays = np.zeros((4, 8), np.float32)
    rays[:, 4:7] = (0.0, 0.0, 4.0)   # toward a point at z = 4 behind the triangle (t = 0.5)
    rays[:, 7] = 1.0 - 2.0 ** -10
    rays[1, 7] = 0.4                 # ends before the triangle
    rays[3, 0:3] = (3.0, 0.0, 0.0)   # passes beside it
    occ, fr = orc.shadow(S, rays, skip=np.array([-1, -1, 0, -1], np.int32))
    assert occ.tolist() == [1, 0, 0, 0] and fr.tolist() == [0, 0, 0, 0]


def _floor_pixels(orc, sc, **kw):
    r = orc.render(orc.Scene(sc), sc.camera, mode="independent", max_bounces=1, tile=(8, 8), debug=True, **kw)
    return r, r["dbg_prim"][0].reshape(sc.camera.height, sc.camera.width)


def test_nee_lambert_floor_in_emitting_box_closed_form(orc):
    """A Lambert floor whose hemisphere is all emitter reflects albedo * le: exactly per
    sample without NEE, and on average (within 4 standard errors) with one light sample."""
    alb = np.float32([0.6, 0.5, 0.4]).astype(np.float64)
    sc = scenes.emitter_box(le=(1.0, 1.0, 1.0), width=16, height=16)
    plain, prim = _floor_pixels(orc, sc, spp=1, seed=1)
    floor = (prim == 8) | (prim == 9)
    assert floor.mean() > 0.3
    assert np.array_equal(plain["rgb"][floor], np.broadcast_to(alb, (floor.sum(), 3)))
    spp = 256
    nee, _ = _floor_pixels(orc, sc, spp=spp, seed=1, nee=True)
    r = nee["rgb"][floor]
    assert nee["counters"][3] > 0.9 * floor.sum() * spp
    # each floor pixel's mean has a spread of sigma / sqrt(spp); pool the pixels
    est = r.mean(axis=0)
    se = r.std(axis=0) / np.sqrt(r.shape[0])
    assert (np.abs(est - alb) < 4 * se + 1e-9).all(), (est, alb, se)
    assert (np.abs(est - alb) < 0.03 * alb).all()


@pytest.mark.parametrize("floor,params", [(scenes.MAT_GGX, (0.9, 0.7, 0.4, 0.3)),
                                          (scenes.MAT_LAMBERT, (0.6, 0.5, 0.4, 0.0))])
def test_nee_has_the_mean_of_plain_path_tracing(orc, floor, params):
    """Emitting box with spheres (occlusion; Lambert, GGX and mirror spheres): the per-pixel
    difference between NEE and plain path tracing has zero mean (4 standard errors)."""
    sc = scenes.emitter_box(floor=floor, floor_params=params, n_spheres=12, seed=4, width=24, height=24)
    S = orc.Scene(sc)
    kw = dict(mode="independent", max_bounces=3, tile=(8, 8), spp=64)
    a = orc.render(S, sc.camera, seed=1, **kw)["rgb"].reshape(-1, 3)
    b = orc.render(S, sc.camera, seed=2, nee=True, **kw)["rgb"].reshape(-1, 3)
    d = (b - a).mean(axis=1)
    se = d.std() / np.sqrt(d.size)
    assert abs(d.mean()) < 4 * se, (d.mean(), se)
    assert abs(d.mean()) < 0.02 * a.mean()


def test_nee_changes_nothing_without_emitters_or_at_mirrors(orc):
    sc = scenes.tiny(material_mix="mixed")
    S = orc.Scene(sc)
    kw = dict(mode="direction_reuse", max_bounces=2, tile=(4, 4), k=8, spp=2, seed=3)
    a = orc.render(S, sc.camera, **kw)
    b = orc.render(S, sc.camera, nee=True, **kw)
    assert np.array_equal(a["rgb"], b["rgb"]) and b["counters"][3] == 0
    # a mirror floor: no light sample there, and the emission seen in it still counts
    box = scenes.emitter_box(floor=scenes.MAT_MIRROR, floor_params=(0.9, 0.8, 0.7, 0.0), width=16, height=16)
    c, prim = _floor_pixels(orc, box, spp=1, seed=2)
    d, _ = _floor_pixels(orc, box, spp=1, seed=2, nee=True)
    floor = (prim == 8) | (prim == 9)
    assert floor.mean() > 0.3
    assert np.array_equal(c["rgb"][floor], d["rgb"][floor])
    assert np.allclose(c["rgb"][floor], np.float32([0.9, 0.8, 0.7]))


@pytest.mark.parametrize("alpha", [0.15, 0.4])
def test_ggx_pdf_is_the_sampler_density(orc, alpha):
    """pdf_ggx integrates over the upper hemisphere to the fraction of valid samples of
    sample_ggx, and f cos / pdf reproduces the sampler's weight for every sampled direction."""
    f0 = [0.9, 0.6, 0.3]
    wo = np.float32([np.sin(0.7), 0.0, np.cos(0.7)])
    G = 120
    valid = 0
    for a in range(G):
        for b in range(G):
            ok, wi, wt = orc.sample_ggx(wo, alpha, f0, (a + 0.5) / G, (b + 0.5) / G)
            if not ok:
                continue
            valid += 1
            pdf = orc.pdf_ggx(wo, wi, alpha)
            f = orc.eval_ggx(wo, wi, alpha, f0)
            assert np.allclose(f * wi[2] / pdf, wt, rtol=2e-4), (f * wi[2] / pdf, wt)
    nt, nphi = 500, 400
    mu = (np.arange(nt) + 0.5) / nt
    phi = (np.arange(nphi) + 0.5) / nphi * 2 * np.pi
    mass = 0.0
    for m in mu:
        st = np.sqrt(1 - m * m)
        for ph in phi:
            mass += orc.pdf_ggx(wo, [st * np.cos(ph), st * np.sin(ph), m], alpha)
    mass *= (1.0 / nt) * (2 * np.pi / nphi)
    assert abs(mass - valid / G ** 2) < 0.01, (mass, valid / G ** 2)


def test_nee_lowers_variance_under_a_small_light(orc):
    """A closed box lit by a small ceiling patch: light sampling with MIS has the mean of
    plain path tracing and a clearly lower per-pixel variance."""
    sc = scenes.emitter_box(n_spheres=6, seed=2, width=24, height=24)
    # keep only a 0.4 x 0.4 emitter patch under the ceiling; the walls become Lambert
    tris = np.concatenate([sc.tri_xyz, np.array([[-0.2, 0.999, -0.2, 0.2, 0.999, -0.2, 0.2, 0.999, 0.2],
                                                  [-0.2, 0.999, -0.2, 0.2, 0.999, 0.2, -0.2, 0.999, 0.2]],
                                                 np.float32)])
    mat = np.concatenate([np.where(sc.tri_mat == 1, 2, sc.tri_mat), [1, 1]])
    params = sc.mat_params.copy()
    params[1, 4:7] = 30.0
    small = scenes._finish("small_light", tris, mat, sc.mat_type, params, (0, 0, 0), sc.camera)
    S = orc.Scene(small)
    kw = dict(mode="independent", max_bounces=2, tile=(8, 8), spp=16)
    res = {}
    for nee in (False, True):
        imgs = np.array([orc.render(S, small.camera, seed=s, nee=nee, **kw)["rgb"] for s in (1, 2, 3, 4)])
        res[nee] = (imgs.mean(), imgs.var(axis=0, ddof=1).mean())
    assert abs(res[True][0] - res[False][0]) < 0.05 * res[False][0], res
    assert res[True][1] < 0.5 * res[False][1], res


def test_shared_light_samples(orc):
    """Shared light samples (every member of a group joins the light point of the group's
    first alive member): with one pixel per group they are each pixel's own samples, bit
    for bit; with groups of 16 the image keeps the mean of plain path tracing."""
    sc = scenes.emitter_box(floor=scenes.MAT_GGX, floor_params=(0.9, 0.7, 0.4, 0.3), n_spheres=12, seed=4,
                            width=24, height=24)
    S = orc.Scene(sc)
    kw = dict(mode="independent", max_bounces=3, tile=(4, 4), spp=4, seed=3)
    own = orc.render(S, sc.camera, k=1, nee=True, **kw)
    shared = orc.render(S, sc.camera, k=1, nee=True, nee_shared=True, **kw)
    assert np.array_equal(own["rgb"], shared["rgb"])
    a, b = [], []
    for f in range(24):
        kw = dict(mode="independent", max_bounces=3, tile=(4, 4), k=16, spp=4, seed=5, frame_base=100 * f)
        a.append(orc.render(S, sc.camera, **kw)["rgb"].mean())
        b.append(orc.render(S, sc.camera, nee=True, nee_shared=True, **kw)["rgb"].mean())
    a, b = np.array(a), np.array(b)
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 4 * se, (a.mean(), b.mean(), se)
    assert abs(a.mean() - b.mean()) < 0.02 * a.mean()
