"""Stage-by-stage parity of the GPU path against the oracle in replay mode.

The GPU renders one frame with the replay capture (every trace's ray, hit distance and
throughput).  The oracle then checks each stage on the GPU's own inputs: the closest hit of
every captured ray (Sec. 1's intersection step), and every shading step (Sec. 3.2: shade,
classify, reuse, spawn) recomputed from the captured state of the trace before it, and the
radiance those steps add.  One fragile closest-hit decision exempts only that ray's trace
check; every pixel's shading steps and radiance are still compared."""
import numpy as np
import pytest
import torch

from paper_2310_07182_gb300 import scenes
from replay_util import replay_check, tile_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


_cache = {}


def _pair(cr, orc, name, bvh8=False, **kw):
    key = (name, bvh8, tuple(sorted(kw.items())))
    if key not in _cache:
        sc = getattr(scenes, name)(**kw)
        flags = cr.CR_BVH2 | (cr.CR_BVH8Q if bvh8 else 0)
        _cache[key] = (sc, cr.Scene(sc, bvh_flags=flags), orc.Scene(sc))
    return _cache[key]


@pytest.mark.parametrize("mode", ["independent", "direction_reuse", "morton_sort"])
def test_replay_tiny(cr, orc, mode):
    """The tiny configuration (64x64, 1,024 Lambert triangles over a ground plane, 1 bounce,
    4x4 groups of 16)."""
    sc, S, O = _pair(cr, orc, "tiny")
    _, rep = replay_check(cr, orc, S, O, sc.camera, max_bounces=1, mode=mode, tile=(4, 4), k=16, seed=1,
                          label=f"tiny {mode}")
    assert rep["shade_and_radiance"] == 1.0 and rep["every_stage"] >= 0.99


@pytest.mark.parametrize("tile,k,interleave", [((4, 4), 1, True), ((4, 4), 4, True), ((4, 4), 16, False),
                                               ((8, 4), 8, True), ((8, 8), 64, True), ((16, 16), 256, True)])
def test_replay_mixed_materials(cr, orc, tile, k, interleave):
    """Lambert / GGX / mirror soup, 3 bounces: every category, warp and block shade kernels."""
    sc, S, O = _pair(cr, orc, "tiny", material_mix="mixed", n_soup=3000)
    _, rep = replay_check(cr, orc, S, O, sc.camera, max_bounces=3, tile=tile, k=k, interleave=interleave, seed=7,
                          frame=3, label=f"mixed {tile} K={k}")
    assert rep["shade_and_radiance"] == 1.0 and rep["every_stage"] >= 0.98


@pytest.mark.parametrize("opt", ["world_reuse", "hybrid_donor", "rough_class", "reuse_depth"])
def test_replay_options(cr, orc, opt):
    sc, S, O = _pair(cr, orc, "tiny", material_mix="mixed", n_soup=3000)
    kw = dict(max_bounces=3, tile=(8, 4), k=8, seed=9)
    if opt == "world_reuse":
        kw["mode"] = "world_reuse"
    elif opt == "hybrid_donor":
        kw["hybrid_donor"] = True
    elif opt == "rough_class":
        kw["diffuse_roughness"] = 0.3
    else:
        kw["reuse_depth"] = 1
    replay_check(cr, orc, S, O, sc.camera, label=opt, **kw)


def test_replay_transmission(cr, orc):
    sc, S, O = _pair(cr, orc, "tiny", material_mix="transmissive", n_soup=3000)
    for mode in ("direction_reuse", "independent"):
        replay_check(cr, orc, S, O, sc.camera, max_bounces=6, mode=mode, tile=(4, 4), k=8, seed=4,
                     label=f"transmission {mode}")


@pytest.mark.parametrize("nee,shared", [(False, False), (True, False), (True, True)])
@pytest.mark.parametrize("bvh8", [False, True])
def test_replay_interior(cr, orc, nee, shared, bvh8):
    """The interior (room, 2,000 spheres, ceiling light) at 160x96, 4 bounces, with and
    without next-event estimation, through either BVH layout."""
    sc, S, O = _pair(cr, orc, "interior", bvh8=True, width=160, height=96)
    _, rep = replay_check(cr, orc, S, O, sc.camera, max_bounces=4, tile=(8, 8), k=8, seed=11, frame=2, nee=nee,
                          nee_shared=shared, bvh=cr.CR_BVH8Q if bvh8 else cr.CR_BVH2,
                          label=f"interior nee={nee} shared={shared} bvh8={bvh8}")
    assert rep["every_stage"] >= 0.99


def test_replay_capture_changes_nothing(cr, orc):
    """Rendering with the replay capture gives the image and counts of a render without it."""
    sc, S, O = _pair(cr, orc, "tiny", material_mix="mixed", n_soup=3000)
    kw = dict(spp=1, max_bounces=3, tile=(8, 4), k=8, seed=5)
    a, sa = S.render(stats=True, **kw)
    dbg, _ = cr.debug_buffers(sc.camera.width, sc.camera.height, 3, replay=True)
    b, sb = S.render(stats=True, debug=dbg, **kw)
    assert torch.equal(a, b) and sa["secondary_rays"] == sb["secondary_rays"]


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["direction_reuse", "independent", "morton_sort"])
def test_replay_landscape_full_size(cr, orc, mode):
    """The benchmark's workload and launch configuration (1920x1080 landscape, 2.1M
    triangles, 1 spp, 2 bounces, 8x8 tiles, K = 8): the GPU renders the whole frame with the
    capture, the oracle replays four bands of 96 tiles spread over the image."""
    sc, S, O = _pair(cr, orc, "landscape")
    cam = sc.camera
    nt = (cam.width // 8) * (cam.height // 8)
    plain, _ = S.render(spp=1, max_bounces=2, mode=mode, tile=(8, 8), k=8, seed=0)
    plain = plain.cpu().numpy().reshape(-1, 3)
    for b0 in (nt // 4, nt // 2, 3 * nt // 4, nt - 96):
        # a grid of shared edges at coordinates up to 100: a ray meets an edge within the FP32
        # rounding band (proportional to the coordinates' magnitude) about 5 times in 1,000
        img, rep = replay_check(cr, orc, S, O, cam, max_bounces=2, mode=mode, tile=(8, 8), k=8, seed=0,
                                tiles=(b0, b0 + 96), label=f"landscape {mode} band {b0}", max_fragile=1e-2)
        assert np.array_equal(img, plain)
        assert rep["shade_and_radiance"] == 1.0 and rep["every_stage"] >= 0.98
        assert rep["rays"] > 96 * 64  # secondary rays reached the band


@pytest.mark.slow
@pytest.mark.parametrize("bvh", ["bvh2", "bvh8q"])
def test_replay_interior_full_size(cr, orc, bvh):
    """The dense-interior precision workload (1280x720, 512,014 triangles, 16 spp, 4 bounces,
    direction reuse, 8x8 tiles, K = 8).  Its 16 frames are rendered one by one with the
    capture and replayed on three bands of 48 tiles; their float sum in frame order, times
    1/16, is the 16-spp render bit for bit (the accumulation the render itself does)."""
    sc, S, O = _pair(cr, orc, "interior", bvh8=True)
    cam = sc.camera
    code = cr.CR_BVH2 if bvh == "bvh2" else cr.CR_BVH8Q
    nt = (cam.width // 8) * (cam.height // 8)
    full, _ = S.render(spp=16, max_bounces=4, mode="direction_reuse", tile=(8, 8), k=8, seed=0, bvh=code)
    acc = np.zeros((cam.width * cam.height, 3), np.float32)
    every = []
    for f in range(16):
        b0 = [0, nt // 2, nt - 48][f % 3]
        img, rep = replay_check(cr, orc, S, O, cam, max_bounces=4, tile=(8, 8), k=8, seed=0, frame=f,
                                tiles=(b0, b0 + 48), bvh=code, label=f"interior {bvh} frame {f}")
        acc += img
        every.append(rep["every_stage"])
        assert rep["shade_and_radiance"] == 1.0
    assert np.array_equal(acc * np.float32(1.0 / 16.0), full.cpu().numpy().reshape(-1, 3))
    assert min(every) >= 0.99
    assert tile_mask(cam, (8, 8), (0, 48)).sum() == 48 * 64
