"""Pins for the oracle's FP64 closest-hit search: brute force over every triangle, closed-form
hits, the tie rule, primitive exclusion and fragility flags."""
import numpy as np

from paper_2310_07182_gb300 import scenes


def _scene(tris, mats=None):
    n = len(tris)
    mats = np.zeros(n) if mats is None else mats
    return scenes._finish("t", np.array(tris, dtype=np.float64), mats, [0], np.zeros((1, 7)), (1, 1, 1), None)


def test_bvh_equals_brute_force(orc):
    for sc in (scenes.tiny(seed=1), scenes.tiny(seed=2, n_soup=3000), scenes.furnace()):
        S = orc.Scene(sc)
        for seed in range(3):
            r = scenes.random_rays(seed, 3000)
            a = orc.trace(S, r, use_bvh=True)
            b = orc.trace(S, r, use_bvh=False)
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_closed_form_hits(orc):
    # triangle in the plane z = 2 around the z axis; unit and scaled directions
    S = orc.Scene(_scene([[-1, -1, 2, 1, -1, 2, 0, 1, 2]]))
    rays = np.zeros((3, 8), np.float32)
    rays[0, 4:7] = (0, 0, 1)
    rays[1, 4:7] = (0, 0, 2)                      # |d| = 2: t = 1
    rays[2, 0:3] = (0, 0, 5)
    rays[2, 4:7] = (0, 0, 1)                      # behind the origin: miss
    prim, t, fr = orc.trace(S, rays)
    assert prim.tolist() == [0, 0, -1]
    assert t[0] == 2.0 and t[1] == 1.0
    assert not fr.any()


def test_tie_goes_to_lower_id_and_skip(orc):
    tri = [-1, -1, 2, 1, -1, 2, 0, 1, 2]
    far = [-1, -1, 3, 1, -1, 3, 0, 1, 3]
    S = orc.Scene(_scene([far, tri, tri, tri]))    # three identical triangles at z = 2
    rays = np.zeros((4, 8), np.float32)
    rays[:, 0:3] = (0.1, -0.2, 0)
    rays[:, 4:7] = (0, 0, 1)
    prim, t, fr = orc.trace(S, rays, skip=np.array([-1, 1, 0, 2], np.int32))
    assert prim.tolist() == [1, 2, 1, 1]
    assert (t == 2.0).all()
    assert (fr & 1).all()                         # exact ties are fragile decisions


def test_edge_and_grazing_rays_are_fragile(orc):
    # two triangles sharing the edge x = 0 in the plane z = 2
    S = orc.Scene(_scene([[-1, -1, 2, 0, -1, 2, 0, 1, 2], [0, -1, 2, 1, -1, 2, 0, 1, 2]]))
    rays = np.zeros((3, 8), np.float32)
    rays[:, 4:7] = (0, 0, 1)
    rays[0, 0:3] = (0.0, 0.0, 0.0)               # through the shared edge
    rays[1, 0:3] = (-0.5, -0.2, 0.0)              # well inside the first
    rays[2, 0:3] = (1.0, -1.0 - 1e-7, 0.0)        # grazes a corner from outside
    prim, t, fr = orc.trace(S, rays)
    assert (fr & 1).tolist() == [1, 0, 1]
    assert prim[1] == 0 and prim[0] in (0, 1)


def test_ill_conditioned_t_is_flagged(orc):
    # a triangle seen almost edge-on, and one hit right next to a far-away origin
    S = orc.Scene(_scene([[-1, -1, 2, 1, -1, 2.001, 0, 1, 2], [50, 50, 50.0, 52, 50, 50.0, 51, 52, 50.0]]))
    rays = np.zeros((3, 8), np.float32)
    rays[0, 0:3] = (0.0, 0.0, 0.0)
    rays[0, 4:7] = (0, 0, 1)                      # head-on: well conditioned
    rays[1, 0:3] = (-3.0, 0.0, 2.0004)
    rays[1, 4:7] = (1.0, 0.0, 0.0)               # nearly in the plane of the triangle
    rays[2, 0:3] = (51.0, 51.0, 50.00001)
    rays[2, 4:7] = (0, 0, -1)                     # t ~ 1e-5 at coordinates ~50
    prim, t, fr = orc.trace(S, rays)
    assert prim.tolist() == [0, 0, 1]
    assert fr[0] == 0 and (fr[1] & 2) and (fr[2] & 2)


def test_tiny_scene_fragility_is_rare(orc):
    sc = scenes.tiny()
    S = orc.Scene(sc)
    r = scenes.random_rays(11, 20000)
    prim, t, fr = orc.trace(S, r)
    assert (fr & 1).mean() < 2e-3
    assert 0.5 < (prim >= 0).mean() < 0.95
