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


def test_matches_the_oracle_on_a_sample(cr, orc):
    """Beyond agreeing with cr_trace_rays, the hits agree with the FP64 oracle: ids bit-exact
    except decisions it flags as fragile, t within max(1e-5 t, T_ERR_K terr)."""
    from replay_util import T_ERR_K
    sc = scenes.tiny(seed=3, n_soup=4000)
    S = cr.Scene(sc)
    n = 20000
    rays_np = scenes.random_rays(8, n)
    rng = np.random.default_rng(8)
    skip_np = np.where(rng.random(n) < 0.3, rng.integers(0, sc.n_tri, n), -1).astype(np.int32)
    p, t = _alloc_free_trace(cr, S, torch.from_numpy(rays_np).cuda(), torch.from_numpy(skip_np).cuda())
    p_ref, t_ref, fr, terr = orc.trace_bound(orc.Scene(sc), rays_np, skip_np)
    ok = (fr & 1) == 0
    assert (~ok).mean() < 2e-3
    assert np.array_equal(p[ok], p_ref[ok])
    hit = ok & (p_ref >= 0)
    assert np.all(np.abs(t[hit] - t_ref[hit]) <= np.maximum(1e-5 * t_ref[hit], T_ERR_K * terr[hit]))
    assert np.all(np.isinf(t[ok & (p_ref < 0)]))


def test_a_warm_call_allocates_nothing(cr):
    """The entry point's promise: after the first call on a device (which looks up the
    scratch array's address, and may load the module that holds it), a call changes neither
    the device's free memory nor the torch caching allocator's counters."""
    sc = scenes.tiny(seed=3, n_soup=4000)
    S = cr.Scene(sc)
    n = cr.CR_TRACE_STATIC_MAX_RAYS
    rays = torch.from_numpy(scenes.random_rays(12, n)).cuda()
    prim = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    cr.cr_trace_rays_static(S.handle, rays, None, prim, t)  # first call on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        cr.cr_trace_rays_static(S.handle, rays, None, prim, t)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
    assert int((prim >= 0).sum()) > 0


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
    with pytest.raises(TypeError):  # the binding refuses a host array before calling C
        cr.cr_trace_rays_static(S.handle, host_rays, None, prim[:16], t[:16])
    # and the C entry point refuses host memory by itself
    L = cr.lib()
    st = L.cr_trace_rays_static(S.handle, host_rays.ctypes.data, None, 16, prim.data_ptr(), t.data_ptr(), None)
    assert st == cr.CR_ERR_INVALID_ARG and b"device pointers" in L.cr_last_error()
