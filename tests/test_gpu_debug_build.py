"""The debug build (CR_DEBUG=1, libcr_debug.so): every node, triangle and material index the
traversal, shade and sum kernels use is checked before it is read; a failed check sets the
scene's error word and the call returns CR_ERR_CUDA.  On valid scenes no check fires and
every result equals the normal build's bit for bit.  (Planting a corrupt index in device
memory to see a check fire is not done: in the normal build that would be an out-of-bounds
read.)"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2310_07182_gb300 import scenes

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the same renders and traces, in whichever library this process loaded
WORK = r'''
import numpy as np, torch
from paper_2310_07182_gb300 import binding as cr, scenes

def run():
    out = {"version": np.array([cr.cr_version()])}
    tiny = scenes.tiny(material_mix="mixed", n_soup=3000)
    S = cr.Scene(tiny, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q | cr.CR_BVH4)
    for mode in ("direction_reuse", "independent", "morton_sort"):
        img, _ = S.render(spp=2, max_bounces=3, mode=mode, tile=(8, 4), k=8, seed=4)
        out["tiny_" + mode] = img.cpu().numpy()
    rays = scenes.random_rays(3, 20000)
    for bvh, name in ((cr.CR_BVH2, "bvh2"), (cr.CR_BVH8Q, "bvh8q"), (cr.CR_BVH4, "bvh4")):
        p, t = S.trace(rays, bvh=bvh)
        out["trace_p_" + name], out["trace_t_" + name] = np.asarray(p), np.asarray(t)
        p, t = S.trace(rays, bvh=bvh, any_hit=True)
        out["any_p_" + name] = np.asarray(p)
    interior = scenes.interior(width=160, height=96)
    I = cr.Scene(interior, bvh_flags=cr.CR_BVH2 | cr.CR_BVH8Q | cr.CR_BVH4)
    for bvh, name in ((cr.CR_BVH2, "bvh2"), (cr.CR_BVH8Q, "bvh8q"), (cr.CR_BVH4, "bvh4")):
        img, _ = I.render(spp=3, max_bounces=4, tile=(8, 8), k=8, seed=2, bvh=bvh, nee=True)
        out["interior_nee_" + name] = img.cpu().numpy()
    return out
'''

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[2])
exec(sys.argv[3])
import numpy as np
np.savez(sys.argv[1], **run())
'''


def test_debug_build_changes_nothing_on_valid_scenes(tmp_path):
    from paper_2310_07182_gb300 import build
    lib = build.build(debug=True)
    dst = str(tmp_path / "debug.npz")
    env = dict(os.environ, CR_LIB=lib)
    subprocess.run([sys.executable, "-c", CHILD, dst, ROOT, WORK], env=env, check=True, cwd=ROOT)
    dbg = np.load(dst)
    assert "debug" in str(dbg["version"][0])
    scope = {}
    exec(WORK, scope)
    ref = scope["run"]()
    assert "debug" not in str(ref["version"][0])
    for key, v in ref.items():
        if key == "version":
            continue
        assert np.array_equal(dbg[key], v), key
    assert (ref["trace_p_bvh2"] >= 0).mean() > 0.3 and ref["tiny_direction_reuse"].max() > 0
