"""Batched form: jobs of several scenes, sizes, spp, bounce counts and modes merged into one
wavefront (one launch per stage per bounce), directly or replayed from a CUDA graph.  Every
job's image must equal its stand-alone render bit for bit, because random numbers are keyed
by (pixel, frame, bounce) and every reuse group lies inside one tile of one job."""
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


SPECS = [  # scene, width, height, spp, bounces, mode, seed, frame_base, reuse_depth
    ("tiny", 64, 64, 1, 2, "direction_reuse", 3, 0, 0),
    ("tiny", 37, 53, 3, 1, "independent", 4, 5, 0),
    ("furnace", 48, 32, 2, 3, "direction_reuse", 5, 0, 0),
    ("interior", 96, 64, 2, 4, "direction_reuse", 6, 2, 1),
    ("tiny", 80, 24, 1, 3, "morton_sort", 7, 0, 0),
    ("interior", 40, 40, 3, 2, "independent", 8, 1, 0),
]


@pytest.mark.parametrize("tile,k,interleave,bvh,flags", [((8, 8), 8, True, 1, 0), ((8, 8), 8, True, 1, 1),
                                                         ((4, 4), 4, False, 1, 1), ((16, 16), 64, True, 2, 1),
                                                         ((16, 8), 32, True, 1, 9)])
def test_batch_equals_standalone(cr, world, tile, k, interleave, bvh, flags):
    sc, S = world
    outs, jobs, refs = [], [], []
    for name, w, h, spp, B, mode, seed, fb, depth in SPECS:
        cam = _cam(sc[name].camera, w, h)
        out = torch.full((h, w, 3), -1.0, device="cuda")
        outs.append(out)
        jobs.append(cr.make_job(S[name].handle, cam, out, spp=spp, max_bounces=B, mode=mode, reuse_depth=depth,
                                seed=seed, frame_base=fb))
        ref, _ = S[name].render(cam, spp=spp, max_bounces=B, mode=mode, tile=tile, k=k, interleave=interleave,
                                seed=seed, frame_base=fb, reuse_depth=depth, bvh=bvh)
        refs.append(ref)
    opts = cr.make_batch_opts(tile=tile, k=k, interleave=interleave, bvh=bvh, flags=flags)
    b = cr.cr_batch_create(jobs, opts)
    try:
        for run in range(2):  # a graph replays identically
            for o in outs:
                o.fill_(-1.0)
            st = cr.cr_batch_run(b)
            for o, r in zip(outs, refs):
                assert torch.equal(o, r)
            assert st["secondary_rays"] > 0 and st["kernel_launches"] > 0
    finally:
        cr.cr_batch_destroy(b)


def test_device_bytes_and_autotune(cr, world):
    sc, S = world
    outs = [torch.empty((64, 64, 3), device="cuda") for _ in range(3)]
    jobs = [cr.make_job(S["tiny"].handle, _cam(sc["tiny"].camera, 64, 64), o, spp=1, max_bounces=2, seed=i)
            for i, o in enumerate(outs)]
    opts = cr.make_batch_opts()
    one = cr.cr_batch_device_bytes(jobs[:1], opts)
    three = cr.cr_batch_device_bytes(jobs, opts)
    assert 64 * 64 * 100 < one < three
    rep = cr.cr_batch_autotune(jobs, opts, allow_contiguous=True)
    # every grouping is either timed or rejected by the quality guard; then the stack depth
    assert rep["n_candidates"] + rep["n_rejected"] == 54 + 3
    if any(j.mode == 2 for j in jobs):  # a direction-reuse job: the guard is on
        assert rep["default_mse"] > 0 and rep["best_mse"] <= 1.1 * rep["default_mse"]
    assert rep["best_ms"] <= rep["default_ms"] <= rep["worst_ms"]
    assert opts.group_w in (4, 8, 16) and opts.k <= opts.group_w * opts.group_h // 4
    assert (opts.group_w, opts.k, opts.interleave, opts.block, opts.stack) == (
        rep["best_group_w"], rep["best_k"], rep["best_interleave"], rep["best_block"], rep["best_stack"])
    assert opts.stack in (8, 16, 32)


def test_batch_rejects_bad_jobs(cr, world):
    sc, S = world
    host = np.zeros((8, 8, 3), np.float32)
    j = cr.make_job(S["tiny"].handle, _cam(sc["tiny"].camera, 8, 8), host)
    with pytest.raises(cr.CrError) as ei:
        cr.cr_batch_create([j], cr.make_batch_opts())
    assert "device buffer" in str(ei.value)
    out = torch.empty((8, 8, 3), device="cuda")
    j = cr.make_job(S["tiny"].handle, _cam(sc["tiny"].camera, 8, 8), out, max_bounces=17)
    with pytest.raises(cr.CrError):
        cr.cr_batch_create([j], cr.make_batch_opts())
