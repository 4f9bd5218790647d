"""Pins for the oracle's interleaved grouping (Sec. 3.3) and its counter-based RNG."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            out[k] = [int(x) for x in v]
    return out


def test_lcg_hand_worked(orc):
    g = _read_golden("lcg_m16_a5_c3_x7.txt")
    seq = orc.lcg_sequence(g["m"][0], g["a"][0], g["c"][0], g["x0"][0])
    assert seq.tolist() == g["sigma"]
    assert (seq // 4).tolist() == g["group"]


@pytest.mark.parametrize("tile", [(1, 1), (2, 1), (2, 2), (4, 4), (8, 8), (16, 8), (16, 16), (32, 8)])
def test_sigma_is_permutation_with_equal_groups(orc, tile):
    W, H = tile
    m = W * H
    for t in range(40):
        for f in range(3):
            sigma, (a, c, x0) = orc.tile_sigma(W, H, t, f, seed=12345)
            assert sorted(sigma.tolist()) == list(range(m))  # bijection on [0, m)
            if m >= 4:
                assert a % 4 == 1
            assert c % 2 == 1 and a < max(m, 2) and c < max(m, 2) and x0 < m
            for K in [k for k in (1, 2, 4, 8, 16, 32, 64) if m % k == 0]:
                counts = np.bincount(sigma // K, minlength=m // K)
                assert (counts == K).all()  # every group has exactly K pixels


def test_affine_special_case(orc):
    """a = 1 reduces the sequence to the affine map x_i = x_0 + c i (mod m)."""
    for m in (16, 64, 256):
        for c in (1, 3, 5, m - 1):
            for x0 in (0, 7, m - 1):
                seq = orc.lcg_sequence(m, 1, c, x0)
                assert seq.tolist() == [(x0 + c * i) % m for i in range(m)]


def test_composition_varies_per_tile_and_frame(orc):
    """Sec. 3.3: the group composition changes from tile to tile and from frame to frame."""
    base, _ = orc.tile_sigma(8, 8, 0, 0, seed=1)
    other_tiles = [orc.tile_sigma(8, 8, t, 0, seed=1)[0] for t in range(1, 33)]
    other_frames = [orc.tile_sigma(8, 8, 0, f, seed=1)[0] for f in range(1, 33)]
    assert sum((s != base).any() for s in other_tiles) >= 30
    assert sum((s != base).any() for s in other_frames) >= 30


def test_contiguous_is_identity(orc):
    sigma, abc = orc.tile_sigma(8, 8, 5, 9, seed=3, lcg=False)
    assert sigma.tolist() == list(range(64))


def test_philox_uniform_bits(orc):
    """Each output bit of Philox4x32-10 is fair over 4096 consecutive counters, and the
    24-bit uniforms pass a chi-square test over 64 bins."""
    outs = np.array([orc.philox(0x1234_5678_9ABC, [i, 7, 3, 0x42534446]) for i in range(4096)], dtype=np.uint64)
    bits = ((outs[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    p = bits.mean(axis=0)
    sigma = 0.5 / np.sqrt(outs.shape[0])
    assert np.abs(p - 0.5).max() < 5.5 * sigma
    u = (outs >> 8).astype(np.float64) / 2.0 ** 24
    hist, _ = np.histogram(u.ravel(), bins=64, range=(0, 1))
    exp = u.size / 64
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 120.0  # 63 dof, p ~ 1e-5
    assert len({tuple(r) for r in outs.tolist()}) == outs.shape[0]


def test_philox_key_and_counter_words_all_matter(orc):
    ref = orc.philox(5, [1, 2, 3, 4])
    assert not np.array_equal(ref, orc.philox(6, [1, 2, 3, 4]))
    assert not np.array_equal(ref, orc.philox(5 | (1 << 32), [1, 2, 3, 4]))
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] += 1
        assert not np.array_equal(ref, orc.philox(5, c))
