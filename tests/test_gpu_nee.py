"""Next-event estimation on the GPU against the oracle: shadow-ray visibility (any-hit
traversal) decision by decision, rendered images pixel by pixel (relative 1e-4 outside the
pixels the oracle flags as fragile), shadow-ray counts, and the batched, serving and BVH8-Q
forms bit-identical to stand-alone BVH2 renders."""
import numpy as np
import pytest
import torch

from gpu_util import radiance_close
from paper_2310_07182_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


_cache = {}


def _trio(cr, orc, name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        sc = getattr(scenes, name)(**kw)
        _cache[key] = (sc, cr.Scene(sc, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q), orc.Scene(sc))
    return _cache[key]


def _shadow_rays(sc, n, seed):
    """Rays from random points toward random emitter-free targets, ending at 1 - 2^-10."""
    rng = np.random.default_rng(seed)
    lo, hi = sc.tri_xyz.reshape(-1, 3).min(axis=0), sc.tri_xyz.reshape(-1, 3).max(axis=0)
    o = rng.uniform(lo, hi, size=(n, 3))
    q = rng.uniform(lo, hi, size=(n, 3))
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = (q - o).astype(np.float32)
    rays[:, 7] = 1.0 - 2.0 ** -10
    return rays


@pytest.mark.parametrize("bvh", ["bvh2", "bvh8"])
def test_any_hit_visibility_matches_oracle(cr, orc, bvh):
    sc, S, O = _trio(cr, orc, "tiny", seed=5, n_soup=3000)
    rays = _shadow_rays(sc, 20000, 3)
    skip = np.where(np.arange(len(rays)) % 7 == 0, np.arange(len(rays)) % 3000, -1).astype(np.int32)
    prim, t = S.trace(rays, skip, any_hit=True, bvh=cr.CR_BVH2 if bvh == "bvh2" else cr.CR_BVH8Q)
    prim, t = np.asarray(prim), np.asarray(t)
    occ, fr = orc.shadow(O, rays, skip)
    ok = fr == 0
    assert ok.mean() > 0.999 and 0.1 < occ.mean() < 0.95
    assert ((prim >= 0) == occ.astype(bool))[ok].all()
    # a reported occluder is a real hit before tmax that is not the skipped triangle
    hit = prim >= 0
    assert (t[hit] < rays[hit, 7]).all() and (t[hit] > 0).all()
    assert (prim[hit] != skip[hit]).all()
    assert np.isinf(t[~hit]).all()


def _check(img, ref, max_taint):
    ok = ref["taint"] == 0
    c = ref["counters"]
    print(f"end-to-end: tainted pixels {(~ok).mean():.4f} (bound {max_taint}), fragile decisions "
          f"{int(c[2])} of {int(c[0] + c[1])} rays ({c[2] / max(1, c[0] + c[1]):.2e}), fragile shadow "
          f"decisions {int(c[4])} of {int(c[3])}")
    assert ok.mean() >= 1 - max_taint, f"{(~ok).sum()} tainted pixels"
    good, excess, nbad = radiance_close(img, ref["rgb"], ok)
    assert good, f"{nbad} pixels off by up to {excess} beyond tolerance"


@pytest.mark.parametrize("mode,tile,k", [("independent", (8, 8), 8), ("direction_reuse", (8, 8), 8),
                                         ("direction_reuse", (8, 8), 64), ("morton_sort", (4, 4), 16)])
def test_nee_render_matches_oracle(cr, orc, mode, tile, k):
    """Emitting box with 12 spheres (Lambert, GGX, mirror): occlusion, every material class,
    emitters on five walls."""
    sc, S, O = _trio(cr, orc, "emitter_box", floor=scenes.MAT_GGX, floor_params=(0.9, 0.7, 0.4, 0.3),
                     n_spheres=12, seed=4, width=48, height=40)
    kw = dict(spp=2, max_bounces=3, mode=mode, tile=tile, k=k, seed=7)
    img, st = S.render(stats=True, nee=True, **kw)
    ref = orc.render(O, sc.camera, nee=True, **kw)
    _check(img.cpu().numpy(), ref, max_taint=0.06 if k == 64 else 0.02)  # a fragile ray taints its group
    c = ref["counters"]
    assert c[3] > 0 and abs(int(st["shadow_rays"]) - int(c[3])) <= max(2, int(c[4]) + 1e-3 * c[3])
    assert st["secondary_rays"] == c[1] or abs(int(st["secondary_rays"]) - int(c[1])) <= int(c[2]) * k
    assert st["ms_trace_shadow"] > 0


def test_nee_interior_matches_oracle(cr, orc):
    """The interior (2,000 spheres, small ceiling light) at reduced resolution."""
    sc, S, O = _trio(cr, orc, "interior", width=96, height=64)
    kw = dict(spp=2, max_bounces=3, mode="direction_reuse", tile=(8, 8), k=8, seed=11)
    img, st = S.render(stats=True, nee=True, **kw)
    ref = orc.render(O, sc.camera, nee=True, **kw)
    _check(img.cpu().numpy(), ref, max_taint=0.08)
    assert st["shadow_rays"] > 0.3 * st["secondary_rays"]


def test_nee_without_emitters_is_plain_rendering(cr, orc):
    sc, S, O = _trio(cr, orc, "tiny", material_mix="mixed")
    kw = dict(spp=2, max_bounces=2, mode="direction_reuse", tile=(4, 4), k=8, seed=3)
    a, _ = S.render(**kw)
    b, st = S.render(stats=True, nee=True, **kw)
    assert torch.equal(a, b) and st["shadow_rays"] == 0
    c, _ = S.render(**kw)  # NEE buffers allocated, NEE off again
    assert torch.equal(a, c)


def test_nee_bvh8_batch_and_server_identical(cr, orc):
    sc, S, O = _trio(cr, orc, "emitter_box", floor=scenes.MAT_LAMBERT, floor_params=(0.6, 0.5, 0.4, 0.0),
                     n_spheres=12, seed=4, width=40, height=32)
    kw = dict(spp=2, max_bounces=3, tile=(8, 8), k=8, seed=5)
    a, _ = S.render(mode="direction_reuse", nee=True, **kw)
    b, _ = S.render(mode="direction_reuse", nee=True, bvh=cr.CR_BVH8Q, **kw)
    assert torch.equal(a, b)
    plain, _ = S.render(mode="direction_reuse", **kw)
    assert not torch.equal(a, plain)
    # a batch mixing NEE and plain jobs: each job equals its stand-alone render
    cam = sc.camera
    outs = [torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    jobs = [cr.make_job(S.handle, cam, outs[0], spp=2, max_bounces=3, seed=5, nee=True),
            cr.make_job(S.handle, cam, outs[1], spp=2, max_bounces=3, seed=5, nee=False)]
    b = cr.cr_batch_create(jobs, cr.make_batch_opts(tile=(8, 8), k=8, flags=cr.CR_BATCH_GRAPH))
    try:
        st = cr.cr_batch_run(b)
    finally:
        cr.cr_batch_destroy(b)
    assert torch.equal(outs[0], a) and torch.equal(outs[1], plain)
    assert st["shadow_rays"] > 0
    # the serving loop
    srv = cr.cr_server_create(256 << 20, tile=(8, 8), k=8)
    try:
        out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
        jid = cr.cr_server_submit(srv, cr.make_job(S.handle, cam, out, spp=2, max_bounces=3, seed=5, nee=True))
        cr.cr_server_wait(srv, jid, 60000)
    finally:
        cr.cr_server_destroy(srv)
    assert torch.equal(out, a)


@pytest.mark.parametrize("tile,k", [((8, 8), 8), ((8, 8), 64)])
def test_shared_light_samples_match_oracle(cr, orc, tile, k):
    """One light point per group (drawn from the first alive member's stream): warp and
    block shade kernels against the oracle."""
    sc, S, O = _trio(cr, orc, "emitter_box", floor=scenes.MAT_GGX, floor_params=(0.9, 0.7, 0.4, 0.3),
                     n_spheres=12, seed=4, width=48, height=40)
    kw = dict(spp=2, max_bounces=3, mode="direction_reuse", tile=tile, k=k, seed=7)
    img, st = S.render(stats=True, nee=True, nee_shared=True, **kw)
    ref = orc.render(O, sc.camera, nee=True, nee_shared=True, **kw)
    _check(img.cpu().numpy(), ref, max_taint=0.06 if k == 64 else 0.03)
    own, _ = S.render(nee=True, **kw)
    assert not torch.equal(img, own)
