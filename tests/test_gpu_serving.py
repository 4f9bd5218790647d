"""Serving with continuous batching: requests of several scenes, sizes, spp and bounce counts
submitted while others render; each result must equal its stand-alone render (same tile
shape, K and interleave) bit for bit, alone or in the mix, with host or device outputs."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_2310_07182_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def world(cr):
    sc = {"tiny": scenes.tiny(material_mix="mixed", n_soup=3000), "furnace": scenes.furnace(),
          "interior": scenes.interior(n_spheres=300, width=96, height=64)}
    S = {k: cr.Scene(v, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q) for k, v in sc.items()}
    return sc, S


def _cam(c, w, h):
    return scenes.Camera(c.pos, c.look_at, c.up, c.vfov_deg, w, h)


def _requests(rng, n):
    names = ["tiny", "furnace", "interior"]
    modes = ["direction_reuse", "independent", "morton_sort"]
    out = []
    for i in range(n):
        out.append(dict(name=names[i % 3], w=int(rng.integers(8, 120)), h=int(rng.integers(8, 90)),
                        spp=int(rng.choice([1, 2, 4, 7])), B=int(rng.integers(1, 5)), mode=modes[(i // 3) % 3],
                        seed=int(rng.integers(0, 1000)), fb=int(rng.integers(0, 50))))
    return out


@pytest.mark.parametrize("bvh,express", [(1, 0), (2, 0), (1, 40_000), (2, 40_000)])
def test_results_equal_standalone_in_the_mix(cr, world, bvh, express):
    """With an express lane, the requests of at most 40,000 ray steps (about a third of this
    mix) render in the second wavefront; every result is still its stand-alone render."""
    sc, S = world
    rng = np.random.default_rng(bvh)
    reqs = _requests(rng, 24)
    srv = cr.cr_server_create(512 << 20, tile=(8, 8), k=8, bvh=bvh, express_rays=express)
    try:
        ids, outs = [], []
        for i, r in enumerate(reqs):
            cam = _cam(sc[r["name"]].camera, r["w"], r["h"])
            out = (np.full((r["h"], r["w"], 3), -1, np.float32) if i % 2 else
                   torch.full((r["h"], r["w"], 3), -1.0, device="cuda"))
            outs.append(out)
            j = cr.make_job(S[r["name"]].handle, cam, out, spp=r["spp"], max_bounces=r["B"], mode=r["mode"],
                            seed=r["seed"], frame_base=r["fb"])
            ids.append(cr.cr_server_submit(srv, j))
            if i % 5 == 0:
                time.sleep(0.002)  # requests keep arriving while earlier ones render
        lat = [cr.cr_server_wait(srv, jid, 60000) for jid in ids]
        st = cr.cr_server_get_stats(srv)
        # "passes" counts bounce iterations: a job takes spp (B + 1) + 1 of them alone
        steps = [r["spp"] * (r["B"] + 1) + 1 for r in reqs]
        assert st["jobs_done"] == len(reqs) and st["passes"] >= max(steps)
        assert st["passes"] < sum(steps)  # jobs shared launches
        if express:
            small = [r["w"] * r["h"] * r["spp"] * (r["B"] + 1) <= express for r in reqs]
            assert 0 < sum(small) < len(reqs)
        for r, out, l in zip(reqs, outs, lat):
            cam = _cam(sc[r["name"]].camera, r["w"], r["h"])
            ref, _ = S[r["name"]].render(cam, spp=r["spp"], max_bounces=r["B"], mode=r["mode"], tile=(8, 8), k=8,
                                         seed=r["seed"], frame_base=r["fb"], bvh=bvh)
            got = out if isinstance(out, np.ndarray) else out.cpu().numpy()
            assert np.array_equal(got, ref.cpu().numpy())
            assert l["latency_ms"] >= 0 and l["samples"] == r["spp"]
        with pytest.raises(cr.CrError) as ei:
            cr.cr_server_wait(srv, ids[0], 10)  # already collected
        assert ei.value.status == cr.CR_ERR_NOT_FOUND
    finally:
        cr.cr_server_destroy(srv)


def test_admission_by_footprint(cr, world):
    """A budget that holds only a few jobs at a time still completes all of them (equal to
    their stand-alone renders), and a job larger than the whole budget is refused at
    submission."""
    sc, S = world
    srv = cr.cr_server_create(64 << 20, tile=(8, 8), k=8)  # path state for 3 jobs of 256^2
    try:
        cam = _cam(sc["tiny"].camera, 256, 256)
        outs = [torch.empty((256, 256, 3), device="cuda") for _ in range(6)]
        ids = [cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, cam, o, spp=3, max_bounces=2, seed=i))
               for i, o in enumerate(outs)]
        peak = 0
        while cr.cr_server_get_stats(srv)["jobs_done"] < len(ids):
            peak = max(peak, cr.cr_server_get_stats(srv)["active"])
            time.sleep(0.0005)
        stats = [cr.cr_server_wait(srv, i, 60000) for i in ids]
        assert 1 <= peak <= 3 and all(s["samples"] == 3 for s in stats)
        for i, o in enumerate(outs):
            ref, _ = S["tiny"].render(cam, spp=3, max_bounces=2, tile=(8, 8), k=8, seed=i)
            assert torch.equal(o, ref)
        big = cr.make_job(S["tiny"].handle, _cam(sc["tiny"].camera, 4096, 4096), torch.empty(1, device="cuda"))
        with pytest.raises(cr.CrError) as ei:
            cr.cr_server_submit(srv, big)
        assert ei.value.status == cr.CR_ERR_OOM
    finally:
        cr.cr_server_destroy(srv)


def test_a_request_joins_between_bounce_launches(cr, world):
    """Continuous batching at bounce granularity: a small request submitted while a large
    many-bounce job renders is admitted within a fraction of one of that job's samples (it
    joins at the next bounce launch instead of waiting for the sample to end), finishes
    first, and equals its stand-alone render."""
    sc, S = world
    srv = cr.cr_server_create(2 << 30, tile=(8, 8), k=8)
    try:
        big_cam = _cam(sc["interior"].camera, 1024, 1024)
        big = torch.empty((1024, 1024, 3), device="cuda")
        spp, B = 48, 16
        bid = cr.cr_server_submit(srv, cr.make_job(S["interior"].handle, big_cam, big, spp=spp, max_bounces=B,
                                                   seed=3))
        time.sleep(0.02)  # the big job is rendering
        small_cam = _cam(sc["tiny"].camera, 32, 32)
        small = torch.empty((32, 32, 3), device="cuda")
        sid = cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, small_cam, small, spp=1, max_bounces=2, seed=5))
        s_st = cr.cr_server_wait(srv, sid, 60000)
        b_st = cr.cr_server_wait(srv, bid, 60000)
        one_sample = (b_st["t_done_ms"] - b_st["t_admit_ms"]) / spp
        assert b_st["t_admit_ms"] < s_st["t_submit_ms"] < b_st["t_done_ms"] - 4 * one_sample
        assert s_st["t_admit_ms"] - s_st["t_submit_ms"] < 0.5 * one_sample
        assert s_st["t_done_ms"] < b_st["t_done_ms"]
        ref, _ = S["tiny"].render(small_cam, spp=1, max_bounces=2, tile=(8, 8), k=8, seed=5)
        assert torch.equal(small, ref)
        ref, _ = S["interior"].render(big_cam, spp=spp, max_bounces=B, tile=(8, 8), k=8, seed=3)
        assert torch.equal(big, ref)
    finally:
        cr.cr_server_destroy(srv)


def test_express_lane_shortens_small_jobs_beside_a_large_one(cr, world):
    """A small request submitted while a large many-bounce job renders: in the main lane it
    takes one bounce step per iteration of the large job's wavefront; in the express lane its
    steps run in their own wavefront on a higher-priority stream.  The same request, with the
    same large job beside it, renders at least twice as fast with the express lane, still
    finishes before the large job, and its output is the same."""
    sc, S = world
    big_cam = _cam(sc["interior"].camera, 1024, 1024)
    small_cam = _cam(sc["tiny"].camera, 64, 64)
    render_ms = {}
    for express in (0, 1 << 20):
        srv = cr.cr_server_create(2 << 30, tile=(8, 8), k=8, express_rays=express)
        try:
            big = torch.empty((1024, 1024, 3), device="cuda")
            bid = cr.cr_server_submit(srv, cr.make_job(S["interior"].handle, big_cam, big, spp=24, max_bounces=16,
                                                       seed=3))
            time.sleep(0.02)  # the big job is rendering
            small = torch.empty((64, 64, 3), device="cuda")
            sid = cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, small_cam, small, spp=4, max_bounces=3,
                                                       seed=5))
            s_st = cr.cr_server_wait(srv, sid, 60000)
            b_st = cr.cr_server_wait(srv, bid, 60000)
            assert s_st["t_done_ms"] < b_st["t_done_ms"]
            render_ms[express] = s_st["t_done_ms"] - s_st["t_admit_ms"]
            ref, _ = S["tiny"].render(small_cam, spp=4, max_bounces=3, tile=(8, 8), k=8, seed=5)
            assert torch.equal(small, ref)
        finally:
            cr.cr_server_destroy(srv)
    print(f"small job render time beside a large one: main lane {render_ms[0]:.2f} ms, "
          f"express lane {render_ms[1 << 20]:.2f} ms")
    assert render_ms[1 << 20] < 0.5 * render_ms[0]


def test_express_lane_fallbacks(cr, world):
    """A request under the express threshold whose tiles exceed the express lane's slots
    runs in the main lane, and the express lane works at the smallest budget; every result is
    its stand-alone render."""
    sc, S = world
    cam_small = _cam(sc["tiny"].camera, 48, 40)
    # 512 MiB: ~2.05M slots of 157 B, an eighth of them (4,007 tiles of 8x8) in the express
    # lane; a 640x640 request has 6,400 tiles but only 409,600 pixels x 1 spp x 2 = 819,200
    # ray steps
    srv = cr.cr_server_create(512 << 20, tile=(8, 8), k=8, express_rays=1 << 20)
    try:
        cam_wide = _cam(sc["tiny"].camera, 640, 640)
        wide = torch.empty((640, 640, 3), device="cuda")
        small = torch.empty((40, 48, 3), device="cuda")
        ids = [cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, cam_wide, wide, spp=1, max_bounces=1, seed=7)),
               cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, cam_small, small, spp=2, max_bounces=2, seed=8))]
        for jid in ids:
            cr.cr_server_wait(srv, jid, 60000)
        ref, _ = S["tiny"].render(cam_wide, spp=1, max_bounces=1, tile=(8, 8), k=8, seed=7)
        assert torch.equal(wide, ref)
        ref, _ = S["tiny"].render(cam_small, spp=2, max_bounces=2, tile=(8, 8), k=8, seed=8)
        assert torch.equal(small, ref)
    finally:
        cr.cr_server_destroy(srv)
    # 64 MiB, the smallest budget: ~256k slots, an express lane of 500 tiles
    srv = cr.cr_server_create(64 << 20, tile=(8, 8), k=8, express_rays=1 << 20)
    try:
        small = torch.empty((40, 48, 3), device="cuda")
        jid = cr.cr_server_submit(srv, cr.make_job(S["tiny"].handle, cam_small, small, spp=2, max_bounces=2, seed=8))
        cr.cr_server_wait(srv, jid, 60000)
        ref, _ = S["tiny"].render(cam_small, spp=2, max_bounces=2, tile=(8, 8), k=8, seed=8)
        assert torch.equal(small, ref)
    finally:
        cr.cr_server_destroy(srv)
