"""GPU closest-hit traversal vs the FP64 oracle on the same fp32 rays: primitive ids bit-exact
except decisions the oracle flags as fragile, t within max(1e-5 t, T_ERR_K terr), terr being
the oracle's FP32 error scale of the winning hit."""
import numpy as np
import pytest
import torch

from paper_2310_07182_gb300 import scenes
from replay_util import T_ERR_K


def _t_close(t, t_ref, terr):
    return np.abs(t - t_ref) <= np.maximum(1e-5 * t_ref, T_ERR_K * terr)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


def _compare(orc, sc, S, rays, skip=None, max_fragile=2e-3, **kw):
    O = orc.Scene(sc)
    p_ref, t_ref, fr, terr = orc.trace_bound(O, rays, skip=skip)
    prim, t = S.trace(rays, skip, **kw)
    prim, t = np.asarray(prim), np.asarray(t)
    ok = (fr & 1) == 0
    print(f"trace {sc.name}: {len(rays)} rays, fragile {(~ok).mean():.2e}, "
          f"ill-conditioned t {((fr & 2) != 0).mean():.2e}")
    assert (~ok).mean() <= max_fragile
    assert np.array_equal(prim[ok], p_ref[ok])
    hit = ok & (p_ref >= 0)
    assert np.all(_t_close(t[hit], t_ref[hit], terr[hit]))
    assert np.all(np.isinf(t[ok & (p_ref < 0)]))
    return prim, t


@pytest.mark.parametrize("n", [1, 31, 1000, 20001])
def test_tiny_random_rays(cr, orc, n):
    sc = scenes.tiny()
    S = cr.Scene(sc)
    rays = scenes.random_rays(n, n)
    _compare(orc, sc, S, rays)
    # device tensors in and out give the same answer
    p1, t1 = S.trace(rays)
    p2, t2 = S.trace(torch.from_numpy(rays).cuda())
    assert np.array_equal(np.asarray(p1), p2.cpu().numpy())
    assert np.array_equal(np.asarray(t1), t2.cpu().numpy())


def test_launch_shapes_agree(cr, orc):
    sc = scenes.tiny(seed=4, n_soup=5000)
    S = cr.Scene(sc)
    rays = scenes.random_rays(9, 30000)
    ref = _compare(orc, sc, S, rays)
    for block in (32, 64, 256, 512):
        for flags in (0, cr.CR_OPT_PERSISTENT, cr.CR_OPT_SPECULATIVE, cr.CR_OPT_PACKET_SECONDARY):
            p, t = S.trace(rays, block=block, flags=flags)
            assert np.array_equal(np.asarray(p), ref[0]) and np.array_equal(np.asarray(t), ref[1])


def test_skip_tmax_axis_aligned_and_ties(cr, orc):
    tri = [-1, -1, 2, 1, -1, 2, 0, 1, 2]
    far = [-1, -1, 3, 1, -1, 3, 0, 1, 3]
    sc = scenes._finish("dup", np.array([far, tri, tri, tri, tri] + [far] * 7), np.zeros(12), [0],
                        np.zeros((1, 7)), (1, 1, 1), None)
    S = cr.Scene(sc)
    rays = np.zeros((6, 8), np.float32)
    rays[:, 0:3] = (0.1, -0.2, 0.0)
    rays[:, 4:7] = (0.0, 0.0, 1.0)  # zero direction components
    rays[:, 7] = np.inf
    rays[4, 7] = 1.5   # tmax before the first triangle
    rays[5, 4:7] = (0.0, 0.0, -1.0)
    skip = np.array([-1, 1, 2, 0, -1, -1], np.int32)
    prim, t = S.trace(rays, skip)
    assert np.asarray(prim).tolist() == [1, 2, 1, 1, -1, -1]
    assert np.asarray(t)[:4].tolist() == [2.0, 2.0, 2.0, 2.0]


def test_watertight_shared_edges(cr, orc):
    """Rays aimed exactly at shared edges and vertices of a closed mesh never slip through."""
    sc = scenes.furnace(subdiv=3)
    S = cr.Scene(sc)
    v = sc.tri_xyz.reshape(-1, 3, 3).astype(np.float64)
    tgt = np.concatenate([(v[:, 0] + v[:, 1]) / 2, v[:, 2]])  # edge midpoints and vertices
    o = np.zeros_like(tgt)
    o[:, :] = tgt * 3.0 + np.array([0.013, -0.007, 0.011])
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((tgt.shape[0], 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = d
    rays[:, 7] = np.inf
    prim, t = S.trace(rays)
    assert (np.asarray(prim) >= 0).all()


@pytest.mark.slow
def test_landscape_full_size_sample(cr, orc):
    """The 2.1M-triangle landscape: camera rays of the bench's 1920x1080 view, traced on the
    GPU in full, a sample of 3000 checked against the oracle."""
    sc = scenes.landscape()
    S = cr.Scene(sc)
    assert S.info["n_tri"] == 2093058 and S.info["depth2"] < 64
    rng = np.random.default_rng(1)
    cam = sc.camera
    n = 1 << 20
    px = rng.integers(0, cam.width, n)
    py = rng.integers(0, cam.height, n)
    th = np.tan(np.radians(cam.vfov_deg) / 2)
    f = np.array(cam.look_at) - np.array(cam.pos)
    f /= np.linalg.norm(f)
    r = np.cross(f, cam.up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    sx = (2 * (px + 0.5) / cam.width - 1) * th * cam.width / cam.height
    sy = (1 - 2 * (py + 0.5) / cam.height) * th
    d = f + sx[:, None] * r + sy[:, None] * u
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = cam.pos
    rays[:, 4:7] = d
    rays[:, 7] = np.inf
    prim, t = S.trace(torch.from_numpy(rays).cuda())
    prim, t = prim.cpu().numpy(), t.cpu().numpy()
    sel = rng.choice(n, 3000, replace=False)
    O = orc.Scene(sc)
    p_ref, t_ref, fr, terr = orc.trace_bound(O, rays[sel])
    ok = (fr & 1) == 0
    print(f"landscape camera rays: fragile {(~ok).mean():.2e} of {len(sel)}")
    # a grid of shared edges at coordinates up to 100 (FP32 rounding band of ~1e-4)
    assert (~ok).mean() < 1e-2
    assert np.array_equal(prim[sel][ok], p_ref[ok])
    hit = ok & (p_ref >= 0)
    assert np.all(_t_close(t[sel][hit], t_ref[hit], terr[hit]))


@pytest.mark.parametrize("layout", ["bvh8q", "bvh4"])
@pytest.mark.parametrize("name", ["tiny", "interior", "furnace"])
def test_wide_bvh_hits_identical_to_bvh2(cr, orc, name, layout):
    """The 8-bit quantised wide BVH only enlarges boxes (conservative rounding), and the
    4-wide BVH keeps the BVH2's boxes and leaves, so closest hits equal the FP32 BVH2's bit
    for bit, on every ray."""
    sc = getattr(scenes, name)() if name != "interior" else scenes.interior(n_spheres=400)
    wide = cr.CR_BVH8Q if layout == "bvh8q" else cr.CR_BVH4
    S = cr.Scene(sc, bvh_flags=cr.CR_BVH2 | wide)
    assert S.info["n_nodes8" if layout == "bvh8q" else "n_nodes4"] > 0
    lo = np.min(sc.tri_xyz.reshape(-1, 3), axis=0)
    hi = np.max(sc.tri_xyz.reshape(-1, 3), axis=0)
    rng = np.random.default_rng(3)
    n = 200000
    o = rng.uniform(lo, hi, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = d
    rays[:, 7] = np.inf
    rays[::7, 7] = rng.uniform(0.01, 1.0, len(rays[::7]))  # some bounded rays
    rays_t = torch.from_numpy(rays).cuda()
    skip = torch.from_numpy(np.where(rng.random(n) < 0.2, rng.integers(0, sc.n_tri, n), -1).astype(np.int32)).cuda()
    p2, t2 = S.trace(rays_t, skip, bvh=cr.CR_BVH2)
    p8, t8 = S.trace(rays_t, skip, bvh=wide)
    assert torch.equal(p2, p8) and torch.equal(t2.view(torch.int32), t8.view(torch.int32))
    assert 0.05 < float((p2 >= 0).float().mean()) < 0.99
    # and against the oracle on a sample of the unbounded rays (the oracle has no tmax)
    unb = np.isinf(rays[:, 7])
    _compare(orc, sc, S, rays[unb][:4000], skip.cpu().numpy()[unb][:4000], bvh=wide)


def test_l2_read_probe(cr):
    """The roofline's L2 roof: a positive finite bandwidth for an L2-resident buffer, and
    argument errors reported as such."""
    gbs = cr.cr_measure_l2_read(48 << 20, 20)
    assert 1000.0 < gbs < 1e6
    with pytest.raises(cr.CrError):
        cr.cr_measure_l2_read(1024, 1)
