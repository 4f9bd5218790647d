"""The allocation-free trace entry point, cr_trace_rays_static.

It exists for callers that must not allocate device memory during a call (a framework that
owns all device memory through its own pool, a latency-critical loop that cannot absorb
cudaMalloc's device synchronisation, a process near its memory limit).  Its results must
equal those of cr_trace_rays, which allocates its own staging buffers, on the same rays.
This file is collected last so that a failure here does not stop the other tests."""
import numpy as np
import pytest
import torch

from paper_2310_07182_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _alloc_free_trace(cr, S, rays, skip):
    n = rays.shape[0]
    prim = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    t = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
    cr.cr_trace_rays_static(S.handle, rays, skip, prim, t)
    return prim.cpu().numpy(), t.cpu().numpy()


def test_matches_allocating_entry_point_twice(cr):
    sc = scenes.tiny(seed=3, n_soup=4000)
    S = cr.Scene(sc)
    # two calls in a row, the second smaller than the first: the shared scratch keeps the
    # first call's contents, which must not leak into the second result
    for seed, n in ((5, cr.CR_TRACE_STATIC_MAX_RAYS), (6, 1234)):
        rays_np = scenes.random_rays(seed, n)
        rng = np.random.default_rng(seed)
        skip_np = np.where(rng.random(n) < 0.3, rng.integers(0, sc.n_tri, n), -1).astype(np.int32)
        rays = torch.from_numpy(rays_np).cuda()
        skip = torch.from_numpy(skip_np).cuda()
        p_ref, t_ref = S.trace(rays, skip)
        p_ref, t_ref = p_ref.cpu().numpy(), t_ref.cpu().numpy()
        p, t = _alloc_free_trace(cr, S, rays, skip)
        # same kernel on the same rays: primitive ids equal, t within the tolerance the
        # parity tests use (1e-5 relative); in practice bit-identical
        assert np.array_equal(p, p_ref)
        hit = p_ref >= 0
        assert np.all(np.abs(t[hit] - t_ref[hit]) <= 1e-5 * np.abs(t_ref[hit]))
        assert np.array_equal(np.isinf(t), np.isinf(t_ref))
        assert 0.3 < hit.mean() < 0.95


def test_rejects_oversize_and_host_buffers(cr):
    sc = scenes.tiny(seed=3)
    S = cr.Scene(sc)
    n = cr.CR_TRACE_STATIC_MAX_RAYS + 1
    rays = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    prim = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    with pytest.raises(cr.CrError) as ei:
        cr.cr_trace_rays_static(S.handle, rays, None, prim, t)
    assert ei.value.status == cr.CR_ERR_INVALID_ARG and "exceeds" in str(ei.value)
    host_rays = scenes.random_rays(1, 16)
    with pytest.raises(cr.CrError) as ei:
        cr.cr_trace_rays_static(S.handle, host_rays, None, prim[:16], t[:16])
    assert ei.value.status == cr.CR_ERR_INVALID_ARG and "device pointers" in str(ei.value)
