"""Edge cases of the GPU path against the oracle: a one-pixel image, a tile larger than the
image, the largest group (K = 256) over ragged border tiles, the deepest paths (16 bounces),
an empty wavefront after the primary trace (every camera ray misses), and empty trace
calls."""
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


def _both(cr, orc, sc, cam, **kw):
    S, O = cr.Scene(sc), orc.Scene(sc)
    img, st = S.render(cam, stats=True, **kw)
    ref = orc.render(O, cam, **kw)
    return img.cpu().numpy(), st, ref


def _check(img, ref, max_taint=0.05):
    ok = ref["taint"] == 0
    c = ref["counters"]
    print(f"end-to-end: tainted pixels {(~ok).mean():.4f} (bound {max_taint}), fragile decisions "
          f"{int(c[2])} of {int(c[0] + c[1])} rays ({c[2] / max(1, c[0] + c[1]):.2e}), fragile shadow "
          f"decisions {int(c[4])} of {int(c[3])}")
    assert ok.mean() >= 1 - max_taint
    good, excess, nbad = radiance_close(img, ref["rgb"], ok)
    assert good, f"{nbad} pixels off by up to {excess}"


@pytest.mark.parametrize("tile,k", [((1, 1), 1), ((8, 8), 8), ((16, 16), 256)])
def test_one_pixel_image(cr, orc, tile, k):
    sc = scenes.tiny(material_mix="mixed")
    c = sc.camera
    cam = scenes.Camera(c.pos, c.look_at, c.up, 10.0, 1, 1)
    img, st, ref = _both(cr, orc, sc, cam, spp=3, max_bounces=2, mode="direction_reuse", tile=tile, k=k, seed=4)
    assert img.shape == (1, 1, 3)
    _check(img, ref, max_taint=1.0)
    assert st["primary_rays"] == 3


def test_largest_group_over_ragged_tiles(cr, orc):
    """16x16 tiles with K = 256 (the block shade kernel) on a 37 x 23 image: every tile is
    partial, so groups have fewer than K members."""
    sc = scenes.tiny(material_mix="mixed", n_soup=3000)
    c = sc.camera
    cam = scenes.Camera(c.pos, c.look_at, c.up, 50.0, 37, 23)
    img, st, ref = _both(cr, orc, sc, cam, spp=2, max_bounces=3, mode="direction_reuse", tile=(16, 16), k=256,
                         seed=6)
    _check(img, ref, max_taint=0.5)  # one fragile ray taints a whole (partial) tile
    assert img.shape == (23, 37, 3)


def test_sixteen_bounces(cr, orc):
    sc = scenes.interior(n_spheres=200, width=48, height=32)
    img, st, ref = _both(cr, orc, sc, sc.camera, spp=1, max_bounces=16, mode="direction_reuse", tile=(8, 8), k=8,
                         seed=3)
    _check(img, ref, max_taint=0.1)
    assert st["secondary_rays"] > 0


@pytest.mark.parametrize("mode", ["direction_reuse", "morton_sort"])
def test_every_camera_ray_misses(cr, orc, mode):
    """Looking away from all geometry: the wavefront is empty after the primary trace and
    every pixel is the environment (under morton_sort the ray sort runs on zero keys)."""
    sc = scenes.tiny()
    cam = scenes.Camera((0.0, 0.0, -3.0), (0.0, 0.0, -10.0), (0.0, 1.0, 0.0), 30.0, 24, 16)
    img, st, ref = _both(cr, orc, sc, cam, spp=2, max_bounces=3, mode=mode, tile=(8, 8), k=8, seed=1)
    assert st["secondary_rays"] == 0 and ref["counters"][1] == 0
    assert (img == 1.0).all() and (ref["rgb"] == 1.0).all()


def test_empty_trace_calls(cr):
    sc = scenes.tiny()
    S = cr.Scene(sc)
    rays = np.zeros((0, 8), np.float32)
    prim, t = S.trace(rays)
    assert len(prim) == 0 and len(t) == 0
    prim, t = S.trace(torch.zeros((0, 8), dtype=torch.float32, device="cuda"), any_hit=True)
    assert prim.numel() == 0
