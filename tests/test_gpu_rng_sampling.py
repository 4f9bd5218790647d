"""GPU parity of the random-number and sampling primitives: Philox blocks, the interleaved
grouping, the polynomial sine/cosine and the BSDF samplers must equal the oracle's bit for
bit; the oracle's Philox is pinned to cuRAND's Philox4_32_10."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import build_curand_helper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


def _ctrs(n, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[:16] = 0
    c[:16, 0] = np.arange(16)
    return np.ascontiguousarray(c)


def test_oracle_philox_matches_curand(orc):
    lib = C.CDLL(build_curand_helper())
    lib.curand_philox_blocks.argtypes = [C.c_uint64, C.c_void_p, C.c_uint32, C.c_void_p]
    for key in (0, 1, 0xDEADBEEF_12345678):
        c = _ctrs(512, key & 0xFFFF)
        c[:, 1] = 0  # keep the word-0/1 offset small (no carries in the offset form)
        out = np.zeros_like(c)
        assert lib.curand_philox_blocks(key, c.ctypes.data, c.shape[0], out.ctypes.data) == 0
        ref = np.array([orc.philox(key, row) for row in c])
        assert np.array_equal(out, ref)


def test_gpu_philox_matches_oracle(cr, orc):
    c = _ctrs(4096, 3)
    for key in (0, 77, 2 ** 40 + 5):
        out = np.zeros_like(c)
        cr.cr_debug_philox(key, c, out)
        ref = np.array([orc.philox(key, row) for row in c[:512]])
        assert np.array_equal(out[:512], ref)


@pytest.mark.parametrize("shape", [(64, 64, 4, 4), (1920, 1080, 8, 8), (37, 23, 8, 8), (50, 30, 16, 16),
                                   (33, 17, 32, 8), (16, 16, 1, 1), (40, 40, 2, 4)])
@pytest.mark.parametrize("interleave", [True, False])
def test_groups_match_oracle(cr, orc, shape, interleave):
    w, h, W, H = shape
    m = W * H
    for frame in (0, 5):
        out = np.zeros(w * h, dtype=np.uint32)
        cr.cr_debug_groups(w, h, W, H, interleave, 99, frame, out)
        ntx = (w + W - 1) // W
        tiles = sorted(set(range(0, ((w + W - 1) // W) * ((h + H - 1) // H), 97)) | {0})
        for tile in tiles[:60]:
            sigma, _ = orc.tile_sigma(W, H, tile, frame, 99, lcg=interleave)
            tx, ty = tile % ntx, tile // ntx
            for i in range(m):
                px, py = tx * W + i % W, ty * H + i // W
                if px < w and py < h:
                    assert out[py * w + px] == tile * m + sigma[i]


def test_sincos_and_samplers_bit_exact(cr, orc):
    rng = np.random.default_rng(8)
    n = 4000
    u = rng.random((n, 2)).astype(np.float32)
    u[:8] = [[0, 0], [0.5, 0.5], [0.999999, 0.0], [0.25, 0.75], [0.5, 0.0], [0, 0.5], [0.75, 0.75], [0.1, 0.9]]
    wo = rng.normal(size=(n, 3))
    wo[:, 2] = np.abs(wo[:, 2])
    wo[::50, 2] *= -1  # some below the surface: invalid
    wo = (wo / np.linalg.norm(wo, axis=1, keepdims=True)).astype(np.float32)
    param = np.concatenate([rng.uniform(0.05, 0.5, (n, 1)), rng.uniform(0.2, 0.8, (n, 3))], axis=1).astype(np.float32)
    wi = np.zeros((n, 3), np.float32)
    wt = np.zeros((n, 3), np.float32)
    valid = np.zeros(n, np.uint8)
    # sine / cosine on [-pi/4, pi/4]
    x = np.linspace(-np.pi / 4, np.pi / 4, n).astype(np.float32)
    ux = np.ascontiguousarray(np.stack([x, np.zeros_like(x)], 1))
    cr.cr_debug_sample(3, n, None, ux, None, wi, wt, valid)
    for i in range(0, n, 7):
        s, c = orc.sincos(x[i])
        assert wi[i, 0].view(np.uint32) == np.float32(s).view(np.uint32)
        assert wi[i, 1].view(np.uint32) == np.float32(c).view(np.uint32)
    # cosine hemisphere
    cr.cr_debug_sample(0, n, None, u, None, wi, wt, valid)
    for i in range(0, n, 3):
        assert (wi[i].view(np.uint32) == orc.sample_cosine(*u[i]).view(np.uint32)).all()
    # GGX
    cr.cr_debug_sample(1, n, wo, u, param, wi, wt, valid)
    for i in range(0, n, 3):
        ok, rwi, rwt = orc.sample_ggx(wo[i], param[i, 0], param[i, 1:4], u[i, 0], u[i, 1])
        assert bool(valid[i]) == ok
        assert (wi[i].view(np.uint32) == rwi.view(np.uint32)).all()
        assert (wt[i].view(np.uint32) == rwt.view(np.uint32)).all()
