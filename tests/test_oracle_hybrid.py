"""Pins of the hybrid-group donor option (an unbiased alternative to the paper's average
glossy direction): diffuse members of a hybrid group share the first diffuse member's own
cosine sample, glossy members keep their own samples, and the image has the mean of
independent sampling."""
import math

import numpy as np

from paper_2310_07182_gb300 import scenes


def test_hybrid_donor_shares_a_diffuse_sample(orc):
    sc = scenes.split_plane(width=32, height=32, left=scenes.MAT_LAMBERT, right=scenes.MAT_GGX, n_strips=4)
    S = orc.Scene(sc)
    kw = dict(spp=1, max_bounces=1, tile=(8, 8), k=16, seed=5, debug=True)
    r = orc.render(S, sc.camera, mode="direction_reuse", hybrid_donor=True, **kw)
    ind = orc.render(S, sc.camera, mode="independent", **kw)
    cat, cls = r["dbg_cat"][0], r["dbg_cls"][0]
    loc = r["dbg_local"][0].reshape(-1, 3)
    hyb = cat == 3
    assert hyb.sum() > 100
    # glossy members of hybrid groups keep their own (independent) samples
    g = hyb & (cls == 2)
    assert np.array_equal(loc[g], ind["dbg_local"][0].reshape(-1, 3)[g])
    # diffuse members of one hybrid group share one direction, and it is one of their own
    # independent cosine samples (the donor's)
    d = hyb & (cls == 1)
    vals = {tuple(v) for v in loc[d]}
    assert len(vals) < d.sum() // 2
    own = {tuple(v) for v in ind["dbg_local"][0].reshape(-1, 3)[d]}
    assert vals <= own


def test_hybrid_donor_is_unbiased_and_the_average_rule_is_not(orc):
    """Paired per-frame differences from independent sampling (same camera rays and seeds)
    on a mixed Lambert/GGX/mirror soup: the donor option has zero mean; the paper's average
    glossy direction for diffuse members shows its bias (reading 5)."""
    sc = scenes.tiny(material_mix="mixed", width=32, height=32)
    S = orc.Scene(sc)
    a, b, c = [], [], []
    for f in range(96):
        kw = dict(spp=1, max_bounces=2, tile=(4, 4), k=16, seed=9, frame_base=f)
        a.append(orc.render(S, sc.camera, mode="independent", **kw)["rgb"].mean())
        b.append(orc.render(S, sc.camera, mode="direction_reuse", hybrid_donor=True, **kw)["rgb"].mean())
        c.append(orc.render(S, sc.camera, mode="direction_reuse", **kw)["rgb"].mean())
    a, b, c = np.array(a), np.array(b), np.array(c)

    def z(x):
        d = x - a
        return d.mean() / (d.std(ddof=1) / math.sqrt(d.size))

    assert abs(z(b)) < 4
    assert z(c) < -2  # the average-direction rule darkens the image measurably
    assert np.abs(a - b).max() > 0
