"""Host checks of the library's BVH builders (no GPU): every triangle in a leaf, every box on
a triangle's root-to-leaf path containing it -- for the BVH8-Q as the kernel decodes its 8-bit
child boxes, for the BVH4 with NaN planes in unused slots -- and the depth / stack bounds the
kernels rely on."""
import numpy as np
import pytest

from paper_2310_07182_gb300 import scenes


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _check(cr, tris):
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    r = cr.cr_debug_bvh_check(tris)
    n = tris.shape[0]
    assert r["covered2"] == n and r["covered8"] == n and r["covered4"] == n
    assert r["violations2"] == 0 and r["violations8"] == 0 and r["violations4"] == 0
    assert r["depth2"] < 62 and r["stack_bound8"] <= 128
    # the BVH4 kernel's stack holds 96 entries; depth4 counts the nodes on a path, depth2 the
    # levels below the BVH2 root, and a 4-wide node spans at least one BVH2 level
    assert r["depth4"] <= r["depth2"] + 1 and r["stack_bound4"] == 3 * r["depth4"] <= 96
    return r


@pytest.mark.parametrize("make", [lambda: scenes.tiny(), lambda: scenes.tiny(seed=9, n_soup=20000),
                                  lambda: scenes.furnace(subdiv=4), lambda: scenes.split_plane(),
                                  lambda: scenes.interior(n_spheres=200)])
def test_scenes(cr, make):
    sc = make()
    r = _check(cr, sc.tri_xyz)
    assert r["n_nodes8"] <= r["n_nodes2"] and r["n_nodes4"] <= r["n_nodes2"]


def test_degenerate_inputs(cr):
    one = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    _check(cr, one)
    _check(cr, np.repeat(one, 5, axis=0))                   # identical triangles
    pts = np.zeros((300, 9), np.float32)                     # all collapsed to one point
    _check(cr, pts)
    rng = np.random.default_rng(0)
    flat = rng.uniform(-1, 1, (5000, 9)).astype(np.float32)
    flat[:, 1::3] = 0.25                                     # a flat sheet (zero extent in y)
    _check(cr, flat)
    big = rng.uniform(-1e4, 1e4, (3000, 9)).astype(np.float32)  # large, overlapping triangles
    _check(cr, big)
    tiny_far = (rng.uniform(-1e-3, 1e-3, (3000, 9)) + 1e5).astype(np.float32)  # tiny, far from origin
    _check(cr, tiny_far)


def test_landscape_full_size(cr):
    r = _check(cr, scenes.landscape().tri_xyz)
    assert r["n_nodes8"] < r["n_nodes2"] / 2
    # up to four children per node (nodes over leaves stay narrower): about half the BVH2's
    # inner nodes and about half its depth
    assert r["n_nodes4"] < 0.55 * r["n_nodes2"] and r["depth4"] < 0.7 * r["depth2"]
