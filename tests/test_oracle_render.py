"""Pins for the oracle's whole path (Sec. 3): white furnace (closed form), the world-space
reuse of Sec. 3.1 failing it (negative control), reductions to independent sampling,
the direction-sharing rules of Sec. 3.2, categories predicted from geometry, statistical
unbiasedness of diffuse reuse, and tile-split / resume equivalences."""
import math

import numpy as np
import pytest

from paper_2310_07182_gb300 import scenes

TAG_BSDF = 0x42534446


def _to_unit(x):
    return np.float32(np.float32(int(x) >> 8) * np.float32(2.0 ** -24))


@pytest.fixture(scope="module")
def furnace(orc):
    sc = scenes.furnace(albedo=(0.5, 0.25, 0.75), width=32, height=32)
    return sc, orc.Scene(sc)


@pytest.mark.parametrize("mode,k,interleave", [("independent", 16, True), ("morton_sort", 16, True),
                                               ("direction_reuse", 1, True), ("direction_reuse", 4, True),
                                               ("direction_reuse", 16, True), ("direction_reuse", 64, False),
                                               ("direction_reuse", 16, False)])
@pytest.mark.parametrize("bounces", [1, 2, 3])
def test_white_furnace_exact(orc, furnace, mode, k, interleave, bounces):
    sc, S = furnace
    W = 8 if k == 64 else 4
    alb = np.float32([0.5, 0.25, 0.75]).astype(np.float64)
    for fb in (0, 1):
        r = orc.render(S, sc.camera, spp=1, max_bounces=bounces, mode=mode,
                       tile=(W, 64 // W if k == 64 else 4), k=k, interleave=interleave, seed=3, frame_base=fb)
        rgb = r["rgb"].reshape(-1, 3)
        hit = (rgb == alb).all(axis=1)  # exactly albedo * env
        miss = (rgb == 1.0).all(axis=1)
        assert (hit | miss).all()
        assert 0.2 < hit.mean() < 0.9
        assert r["taint"].sum() == 0


@pytest.mark.parametrize("hybrid_donor", [False, True])
def test_hybrid_weight_reading_in_a_mixed_furnace(orc, hybrid_donor):
    """Reading of the hybrid rule's weight (Sec. 3.2 gives none): a diffuse member that takes
    the group's average glossy direction weighs it by its own material, f cos / p_cos =
    albedo.  In a mixed furnace that makes every Lambert pixel exactly albedo, in diffuse
    and in hybrid groups alike; glossy members keep their own samples (their pixels equal
    independent sampling's, bit for bit)."""
    sc = scenes.mixed_furnace()
    S = orc.Scene(sc)
    alb = np.float32([0.5, 0.25, 0.75]).astype(np.float64)
    kw = dict(spp=1, max_bounces=1, tile=(4, 4), k=16, seed=5)
    r = orc.render(S, sc.camera, mode="direction_reuse", debug=True, hybrid_donor=hybrid_donor, **kw)
    ind = orc.render(S, sc.camera, mode="independent", debug=True, **kw)
    cls, cat = r["dbg_cls"][0], r["dbg_cat"][0]
    rgb = r["rgb"].reshape(-1, 3)
    lam = cls == 1
    hybrid_lam = lam & (cat == 3)
    assert hybrid_lam.sum() > 100
    assert (rgb[lam] == alb).all()
    glossy = cls == 2
    assert glossy.sum() > 20
    assert np.array_equal(rgb[glossy], ind["rgb"].reshape(-1, 3)[glossy])
    assert r["taint"].sum() == 0


def test_world_space_reuse_fails_furnace(orc, furnace):
    """Sec. 3.1: reusing a world-space direction sends some rays below the surface; the
    furnace detects it (the test that the tangent-space method passes)."""
    sc, S = furnace
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="world_reuse", tile=(8, 8), k=64, seed=3)
    rgb = r["rgb"].reshape(-1, 3)
    alb = np.float32([0.5, 0.25, 0.75]).astype(np.float64)
    ok = (rgb == alb).all(axis=1) | (rgb == 1.0).all(axis=1)
    assert (~ok).sum() > 20


def _render_pair(orc, sc, S, **kw):
    a = orc.render(S, sc.camera, mode="independent", **kw)
    b = orc.render(S, sc.camera, mode="direction_reuse", **kw)
    return a, b


def test_k1_reuse_equals_independent(orc):
    sc = scenes.tiny(material_mix="mixed")
    S = orc.Scene(sc)
    a, b = _render_pair(orc, sc, S, spp=2, max_bounces=3, tile=(4, 4), k=1, seed=9)
    assert np.array_equal(a["accum"], b["accum"])


def test_all_glossy_reuse_equals_independent(orc):
    sc = scenes.tiny(material_mix="glossy")
    S = orc.Scene(sc)
    a, b = _render_pair(orc, sc, S, spp=1, max_bounces=3, tile=(4, 4), k=16, seed=2)
    assert np.array_equal(a["accum"], b["accum"])


def test_diffuse_groups_share_the_donor_direction(orc):
    """Sec. 3.2 diffuse group: all members' tangent-space exit directions are bit-identical and
    equal the cosine sample drawn from the stream of the member with the smallest shuffled
    number."""
    sc = scenes.tiny()
    S = orc.Scene(sc)
    W = H = 4
    K = 8
    seed, frame = 17, 0
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="direction_reuse", tile=(W, H), k=K, seed=seed,
                   debug=True)
    w = sc.camera.width
    ntx = w // W
    checked = 0
    for tile in range(ntx * (sc.camera.height // H)):
        sigma, _ = orc.tile_sigma(W, H, tile, frame, seed)
        tx, ty = tile % ntx, tile // ntx
        pix = np.array([(ty * H + i // W) * w + tx * W + i % W for i in range(W * H)])
        for g in range(W * H // K):
            mem = pix[np.argsort(sigma)][g * K:(g + 1) * K]  # members in shuffled order
            alive = (r["dbg_flags"][0, mem] & 1).astype(bool)
            if not alive.any():
                continue
            assert (r["dbg_cat"][0, mem] == 1).all()
            loc = r["dbg_local"][0, mem[alive]]
            donor = mem[alive][0]
            h = orc.philox(seed, [donor, frame, 1, TAG_BSDF])
            expect = orc.sample_cosine(_to_unit(h[0]), _to_unit(h[1]))
            assert (loc.view(np.uint32) == expect.view(np.uint32)).all()
            checked += 1
    assert checked > 300


def test_hybrid_groups_take_normalised_glossy_sum(orc):
    """Sec. 3.2 hybrid group: diffuse members take the normalised tangent-space sum of the valid
    glossy/specular exit directions (pairwise over the group's shuffled slots); glossy members
    keep their own sample."""
    sc = scenes.tiny(material_mix="mixed", n_soup=2000)
    S = orc.Scene(sc)
    W = H = 8
    K = 16
    seed = 4
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="direction_reuse", tile=(W, H), k=K, seed=seed,
                   debug=True)
    ind = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="independent", tile=(W, H), k=K, seed=seed,
                     debug=True)
    w = sc.camera.width
    ntx = w // W
    n_hybrid = 0
    for tile in range(ntx * (sc.camera.height // H)):
        sigma, _ = orc.tile_sigma(W, H, tile, 0, seed)
        tx, ty = tile % ntx, tile // ntx
        pix = np.array([(ty * H + i // W) * w + tx * W + i % W for i in range(W * H)])
        for g in range(W * H // K):
            mem = pix[np.argsort(sigma)][g * K:(g + 1) * K]
            if r["dbg_cat"][0, mem[0]] != 3:
                continue
            fl, cl = r["dbg_flags"][0, mem], r["dbg_cls"][0, mem]
            gl = (fl & 2).astype(bool) & (cl == 2)
            v = np.where(gl[:, None], ind["dbg_local"][0, mem], np.float32(0)).astype(np.float32)
            while v.shape[0] > 1:
                v = (v[0::2] + v[1::2]).astype(np.float32)
            v = v[0]
            l = np.sqrt(np.float32((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]))
            dif = ((fl & 1).astype(bool)) & (cl == 1)
            if l > 0:
                u = (v / l).astype(np.float32)
            else:  # no valid glossy sample: the first diffuse member's own sample
                u = ind["dbg_local"][0, mem[dif][0]]
            assert (r["dbg_local"][0, mem[dif]].view(np.uint32) == u.view(np.uint32)).all()
            glossy = (cl == 2)
            assert (r["dbg_local"][0, mem[glossy]].view(np.uint32) ==
                    ind["dbg_local"][0, mem[glossy]].view(np.uint32)).all()
            n_hybrid += 1
    assert n_hybrid > 10


def _strip_plane(width, edges, tx):
    """Plane z=0 cut into vertical strips whose edges fall on pixel-column edges of a camera at
    z=-2 looking +z (column c spans x in [2(1-2(c+1)/w)tx, 2(1-2c/w)tx])."""
    tris, mats = [], []
    xs = [2.0 * (1.0 - 2.0 * c / width) * tx for c in edges]
    xs[0], xs[-1] = 4.0, -4.0
    for s in range(len(xs) - 1):
        x0, x1 = xs[s + 1], xs[s]
        a, b, c, d = (x0, -4.0, 0.0), (x1, -4.0, 0.0), (x1, 4.0, 0.0), (x0, 4.0, 0.0)
        tris += [a + b + c, a + c + d]
        mats += [s % 2, s % 2]
    params = np.zeros((2, 7))
    params[:, 0:3] = [[0.6, 0.5, 0.4], [0.7, 0.7, 0.7]]
    params[:, 3] = 0.3
    cam = scenes.Camera((0.0, 0.0, -2.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, width)
    return scenes._finish("strips", np.array(tris), np.array(mats), [scenes.MAT_LAMBERT, scenes.MAT_GGX], params,
                          (1.0, 1.0, 1.0), cam)


def test_categories_follow_geometry(orc):
    """Groups whose pixels all see the Lambert strips are diffuse, all-GGX groups glossy, mixed
    groups hybrid (Sec. 3.2), with membership from the interleaved grouping (Sec. 3.3)."""
    w, W, H, K, seed = 32, 8, 8, 8, 6
    edges = [0, 8, 16, 19, 32]
    sc = _strip_plane(w, edges, math.tan(math.radians(30.0)))
    S = orc.Scene(sc)
    r = orc.render(S, sc.camera, spp=1, max_bounces=1, mode="direction_reuse", tile=(W, H), k=K, seed=seed,
                   debug=True)
    strip_of_col = np.searchsorted(edges, np.arange(w), side="right") - 1
    col_cls = np.where(strip_of_col % 2 == 0, 1, 2)
    cats = set()
    for tile in range((w // W) ** 2):
        sigma, _ = orc.tile_sigma(W, H, tile, 0, seed)
        tx, ty = tile % (w // W), tile // (w // W)
        cols = np.array([tx * W + i % W for i in range(W * H)])
        pix = np.array([(ty * H + i // W) * w + tx * W + i % W for i in range(W * H)])
        for g in range(W * H // K):
            sel = (sigma // K) == g
            cl = set(col_cls[cols[sel]].tolist())
            expect = 3 if cl == {1, 2} else (1 if cl == {1} else 2)
            if (r["dbg_flags"][0, pix[sel]] & 4).any():
                continue  # a fragile decision (ray exactly on a strip edge)
            assert (r["dbg_cls"][0, pix[sel]] == col_cls[cols[sel]]).all()
            assert (r["dbg_cat"][0, pix[sel]] == expect).all()
            cats.add(expect)
    assert cats == {1, 2, 3}


def test_diffuse_reuse_is_unbiased(orc):
    """Sec. 3.2: reusing a tangent-space direction within a diffuse group keeps importance
    sampling valid, so the expected image equals independent sampling's."""
    sc = scenes.tiny()
    S = orc.Scene(sc)
    means = {"independent": [], "direction_reuse": []}
    for f in range(48):
        for mode in means:
            r = orc.render(S, sc.camera, spp=1, max_bounces=2, mode=mode, tile=(4, 4), k=16, seed=77,
                           frame_base=f)
            means[mode].append(r["rgb"].mean())
    a, b = np.array(means["independent"]), np.array(means["direction_reuse"])
    se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 5 * se
    # and the reuse images really differ from independent ones (correlated sampling)
    assert np.abs(a - b).max() > 0


def test_tile_split_and_resume(orc):
    sc = scenes.tiny(material_mix="mixed")
    S = orc.Scene(sc)
    kw = dict(max_bounces=2, mode="direction_reuse", tile=(4, 4), k=4, seed=5)
    full = orc.render(S, sc.camera, spp=4, **kw)
    nt = (64 // 4) ** 2
    a = orc.render(S, sc.camera, spp=4, tiles=(0, nt // 2 + 3), **kw)
    b = orc.render(S, sc.camera, spp=4, tiles=(nt // 2 + 3, nt), **kw)
    assert np.array_equal(full["accum"], a["accum"] + b["accum"])
    acc = np.zeros_like(full["accum"])
    orc.render(S, sc.camera, spp=2, frame_base=0, accum=acc, **kw)
    orc.render(S, sc.camera, spp=2, frame_base=2, accum=acc, **kw)
    assert np.array_equal(full["accum"], acc)
    one = orc.render(S, sc.camera, spp=4, threads=1, **kw)
    assert np.array_equal(full["accum"], one["accum"])


def test_roughness_threshold_puts_rough_ggx_in_diffuse_groups(orc):
    """The roughness knob of the classes (Sec. 3.2 classifies by material; the threshold is
    a reading): with diffuse_roughness = 0.25 every GGX point of roughness >= 0.25 is in the
    diffuse class, and the alive members of a diffuse group all take the donor's
    tangent-space direction, which lies in the upper hemisphere (a cosine sample)."""
    sc = scenes.tiny(material_mix="mixed", n_soup=3000)
    S = orc.Scene(sc)
    kw = dict(spp=1, max_bounces=1, tile=(4, 4), k=16, seed=9, debug=True)
    r = orc.render(S, sc.camera, mode="direction_reuse", diffuse_roughness=0.25, **kw)
    r0 = orc.render(S, sc.camera, mode="direction_reuse", **kw)
    prim = r["dbg_prim"][0]
    hit = prim >= 0
    mat = sc.tri_mat[prim[hit]]
    ty = sc.mat_type[mat]
    rough = sc.mat_params[mat, 3]
    cls = r["dbg_cls"][0][hit]
    assert (cls[(ty == scenes.MAT_GGX) & (rough >= 0.25)] == 1).all()
    assert (cls[(ty == scenes.MAT_GGX) & (rough < 0.25)] == 2).all()
    assert (r0["dbg_cls"][0][hit][ty == scenes.MAT_GGX] == 2).all()
    # more diffuse groups than with classes by type only
    assert (r["dbg_cat"][0] == 1).sum() > (r0["dbg_cat"][0] == 1).sum()
    w = sc.camera.width
    ntx = w // 4
    loc = r["dbg_local"][0]
    n_checked = 0
    for tile in range(ntx * (sc.camera.height // 4)):
        sigma, _ = orc.tile_sigma(4, 4, tile, 0, 9)
        tx, ty_ = tile % ntx, tile // ntx
        pix = np.array([(ty_ * 4 + i // 4) * w + tx * 4 + i % 4 for i in range(16)])
        mem = pix[np.argsort(sigma)]
        if r["dbg_cat"][0, mem[0]] != 1:
            continue
        alive = (r["dbg_flags"][0, mem] & 1).astype(bool)
        d = loc[mem[alive]]
        assert (d.view(np.uint32) == d[0].view(np.uint32)).all() and d[0, 2] >= 0
        n_checked += 1
    assert n_checked > 20


def test_roughness_threshold_keeps_independent_sampling_and_is_unbiased(orc):
    """The knob changes only how reused directions are drawn: independent sampling is the
    same image bit for bit, and reuse with rough GGX in diffuse groups (cosine samples,
    weight pi f) has independent sampling's mean (hybrid groups use the unbiased donor rule
    here so that only the knob is tested)."""
    sc = scenes.tiny(material_mix="mixed")
    S = orc.Scene(sc)
    kw = dict(spp=1, max_bounces=2, tile=(4, 4), k=16, seed=31)
    a = orc.render(S, sc.camera, mode="independent", **kw)
    b = orc.render(S, sc.camera, mode="independent", diffuse_roughness=0.25, **kw)
    assert np.array_equal(a["rgb"], b["rgb"])
    means = {"independent": [], "direction_reuse": []}
    for f in range(48):
        for mode in means:
            r = orc.render(S, sc.camera, spp=1, max_bounces=2, mode=mode, tile=(4, 4), k=16, seed=77,
                           frame_base=f, diffuse_roughness=0.25, hybrid_donor=True)
            means[mode].append(r["rgb"].mean())
    x, y = np.array(means["independent"]), np.array(means["direction_reuse"])
    se = math.sqrt(x.var(ddof=1) / x.size + y.var(ddof=1) / y.size)
    assert abs(x.mean() - y.mean()) < 5 * se


def test_cosine_sampled_rough_ggx_has_the_directional_albedo(orc):
    """A rough GGX plane in a unit environment, one bounce: each pixel is the weight of its
    direction, so its mean over samples is the directional albedo (integral of f cos),
    whether the direction is GGX-sampled (independent) or a cosine sample weighted pi f (the
    roughness knob).  Both means agree within three standard errors (about 1%), which a
    weight off by a few percent fails."""
    sc = scenes.split_plane(width=16, height=16, left=scenes.MAT_GGX, right=scenes.MAT_GGX)
    sc.mat_params[:, 3] = 0.4
    S = orc.Scene(sc)
    # K = 1: every point draws its own direction, so the pixels' samples are independent
    kw = dict(spp=1, max_bounces=1, tile=(4, 4), k=1, seed=3, diffuse_roughness=0.3)
    per_frame = {"independent": [], "direction_reuse": []}
    for f in range(128):
        for mode in per_frame:
            r = orc.render(S, sc.camera, mode=mode, frame_base=f, debug=True, **kw)
            assert (r["dbg_cls"][0] == 1).all()  # the class label; only reuse changes sampling
            per_frame[mode].append(r["rgb"][..., 0].ravel())
    x, y = np.array(per_frame["independent"]), np.array(per_frame["direction_reuse"])
    se = math.sqrt(x.var() / x.size + y.var() / y.size) / y.mean()
    assert se < 0.005
    assert abs(x.mean() / y.mean() - 1.0) < 3 * se
    # the two estimators really differ sample by sample (cosine vs GGX directions)
    assert not np.array_equal(x, y)


def test_rough_members_of_hybrid_groups_keep_their_own_cosine_sample(orc):
    """Under the paper's hybrid rule the Lambert members take the glossy average, but a
    rough GGX member of the diffuse class keeps its own cosine sample (weighing the average
    by pi f, near its own specular peak, would add energy): its direction equals the one it
    draws alone (K = 1)."""
    sc = scenes.tiny(material_mix="mixed", n_soup=3000)
    S = orc.Scene(sc)
    kw = dict(spp=1, max_bounces=1, seed=9, debug=True, diffuse_roughness=0.25, mode="direction_reuse")
    r = orc.render(S, sc.camera, tile=(4, 4), k=16, **kw)
    alone = orc.render(S, sc.camera, tile=(4, 4), k=1, **kw)
    prim = r["dbg_prim"][0]
    hit = prim >= 0
    mat = np.full(prim.shape, -1)
    mat[hit] = sc.tri_mat[prim[hit]]
    rough = hit & (sc.mat_type[np.maximum(mat, 0)] == scenes.MAT_GGX) & (sc.mat_params[np.maximum(mat, 0), 3] >= 0.25)
    fl, cls = r["dbg_flags"][0], r["dbg_cls"][0]
    w = sc.camera.width
    ntx = w // 4
    n = 0
    for tile in range(ntx * (sc.camera.height // 4)):
        sigma, _ = orc.tile_sigma(4, 4, tile, 0, 9)
        tx, ty = tile % ntx, tile // ntx
        mem = np.array([(ty * 4 + i // 4) * w + tx * 4 + i % 4 for i in range(16)])[np.argsort(sigma)]
        # hybrid groups whose glossy average exists (a valid glossy/specular sample)
        if r["dbg_cat"][0, mem[0]] != 3 or not ((cls[mem] == 2) & ((fl[mem] & 2) == 2)).any():
            continue
        sel = mem[rough[mem] & ((fl[mem] & 1) == 1)]
        assert np.array_equal(r["dbg_local"][0][sel].view(np.uint32), alone["dbg_local"][0][sel].view(np.uint32))
        n += len(sel)
    assert n > 20
