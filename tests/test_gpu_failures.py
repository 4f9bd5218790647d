"""Failure paths that need a GPU but never fault it: bounded waits that run out, requests
larger than the device budget, resumed progressive rendering, invalid renders rejected
before any launch."""
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


def test_server_wait_times_out_then_completes(cr):
    sc = scenes.interior(n_spheres=400, width=256, height=256)
    S = cr.Scene(sc)
    srv = cr.cr_server_create(256 << 20)
    try:
        out = torch.empty((256, 256, 3), device="cuda")
        jid = cr.cr_server_submit(srv, cr.make_job(S.handle, sc.camera, out, spp=64, max_bounces=4))
        with pytest.raises(cr.CrError) as ei:
            cr.cr_server_wait(srv, jid, 0)
        assert ei.value.status == cr.CR_ERR_TIMEOUT
        assert cr.cr_server_poll(srv, jid) is None  # still busy
        st = cr.cr_server_wait(srv, jid, 120000)
        assert st["samples"] == 64
        with pytest.raises(cr.CrError) as ei:
            cr.cr_server_poll(srv, 12345)
        assert ei.value.status == cr.CR_ERR_NOT_FOUND
    finally:
        cr.cr_server_destroy(srv)


def test_resume_progressive_rendering(cr):
    """Samples are keyed by frame index, so 2 + 2 samples resumed at frame_base 2 average to
    the 4-sample render (up to the order of the float sums)."""
    sc = scenes.tiny(material_mix="mixed")
    S = cr.Scene(sc)
    kw = dict(max_bounces=3, tile=(4, 4), k=8, seed=5)
    full, _ = S.render(spp=4, frame_base=0, **kw)
    a, _ = S.render(spp=2, frame_base=0, **kw)
    b, _ = S.render(spp=2, frame_base=2, **kw)
    assert torch.allclose((a + b) / 2, full, rtol=1e-6, atol=1e-7)


def test_invalid_render_arguments(cr):
    sc = scenes.tiny()
    S = cr.Scene(sc)
    out = torch.empty((64, 64, 3), device="cuda")
    for kw, msg in ((dict(tile=(3, 4)), "power of two"), (dict(tile=(4, 4), k=32), "K="),
                    (dict(max_bounces=0), "max_bounces"), (dict(spp=0), "spp"), (dict(bvh=2), "bvh")):
        args = dict(spp=1, max_bounces=1, tile=(4, 4))
        args.update(kw)
        with pytest.raises(cr.CrError) as ei:
            S.render(out=out, **args)
        assert ei.value.status == cr.CR_ERR_INVALID_ARG and msg in str(ei.value)
    bad = scenes.Camera((0, 0, 0), (0, 1, 0), (0, 1, 0), 60.0, 8, 8)  # up parallel to view
    with pytest.raises(cr.CrError):
        S.render(bad, out=torch.empty((8, 8, 3), device="cuda"))


def test_diffuse_reuse_unbiased_on_gpu(cr):
    """Sec. 3.2: tangent-space reuse in all-diffuse groups keeps the expectation; the mean
    image over 96 frames matches independent sampling's within 5 standard errors."""
    sc = scenes.tiny()
    S = cr.Scene(sc)
    means = {}
    for mode in ("independent", "direction_reuse"):
        v = []
        for f in range(96):
            img, _ = S.render(spp=1, max_bounces=2, mode=mode, tile=(4, 4), k=16, seed=77, frame_base=f)
            v.append(float(img.mean()))
        means[mode] = np.array(v)
    a, b = means["independent"], means["direction_reuse"]
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 5 * se
