"""CPU checks of the C-ABI library: it builds, loads, exports every entry point declared in
include/cr.h, and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


def _declared():
    hdr = open(os.path.join(ROOT, "include", "cr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:cr_status|const char\*)\s+(cr_\w+)\s*\(", hdr, re.M)))


def test_exports_every_declared_symbol(cr):
    names = _declared()
    assert len(names) >= 12
    L = C.CDLL(cr.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(cr.exported_names()) == names


def test_struct_layouts(cr):
    assert C.sizeof(cr.cr_material) == 32
    assert C.sizeof(cr.cr_camera) == 48
    assert C.sizeof(cr.cr_render_opts) == 80
    assert C.sizeof(cr.cr_debug) == 72


def test_struct_layouts_match_the_header(cr, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C compiler
    gives the declaration in include/cr.h."""
    import subprocess
    names = ["cr_material", "cr_env", "cr_scene_info", "cr_camera", "cr_stats", "cr_debug", "cr_job",
             "cr_batch_opts", "cr_tune_report", "cr_server_opts", "cr_job_stats", "cr_server_stats",
             "cr_render_opts", "cr_bvh_report"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cr.h"', "int main(void) {"]
    expect = []
    for n in names:
        cls = getattr(cr, n)
        lines.append(f'printf("%zu\\n", sizeof({n}));')
        expect.append(C.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({n}, {f}));')
            expect.append(getattr(cls, f).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_version(cr):
    assert "sm_103a" in cr.cr_version()


def test_invalid_arguments_rejected_without_gpu(cr):
    L = cr.lib()
    out = C.c_void_p()
    m = (cr.cr_material * 1)()
    tris = np.zeros((1, 9), np.float32)
    mats = np.zeros(1, np.uint32)
    assert L.cr_scene_create(None, 0, None, None, 0, None, 1, C.byref(out)) == cr.CR_ERR_INVALID_ARG
    assert b"NULL" in L.cr_last_error()
    assert L.cr_scene_create(tris.ctypes.data, 0, mats.ctypes.data, C.addressof(m), 1, None, 1,
                             C.byref(out)) == cr.CR_ERR_INVALID_ARG
    bad = tris.copy()
    bad[0, 4] = np.nan
    assert L.cr_scene_create(bad.ctypes.data, 1, mats.ctypes.data, C.addressof(m), 1, None, 1,
                             C.byref(out)) == cr.CR_ERR_INVALID_ARG
    assert b"not finite" in L.cr_last_error()
    badm = np.array([3], np.uint32)
    assert L.cr_scene_create(tris.ctypes.data, 1, badm.ctypes.data, C.addressof(m), 1, None, 1,
                             C.byref(out)) == cr.CR_ERR_INVALID_ARG
    cam = cr.cr_camera()
    assert L.cr_render(None, C.byref(cam), 1, 1, 2, 8, 8, None) == cr.CR_ERR_INVALID_ARG
    o = cr.cr_render_opts()
    assert L.cr_render_opts_default(C.byref(o)) == cr.CR_OK
    assert o.interleave == 1 and o.bvh == cr.CR_BVH2 and o.k == 0
    assert L.cr_debug_groups(16, 16, 3, 4, 1, 0, 0, None) == cr.CR_ERR_INVALID_ARG
    assert L.cr_debug_sample(7, 1, None, None, None, None, None, None) == cr.CR_ERR_INVALID_ARG


def test_static_trace_argument_checks_without_gpu(cr):
    """cr_trace_rays_static's binding refuses buffers the C side could overrun (it sees raw
    pointers only): wrong shape, dtype or length, non-contiguous, non-tensor, host tensors."""
    import torch
    ok = dict(rays=torch.zeros((16, 8)), skip=None, prim=torch.zeros(16, dtype=torch.int32),
              t=torch.zeros(16))
    cases = [
        (dict(rays=np.zeros((16, 8), np.float32)), TypeError, "torch tensor"),
        (dict(rays=torch.zeros((16, 7))), ValueError, "shape"),
        (dict(rays=torch.zeros(128)), ValueError, "shape"),
        (dict(rays=torch.zeros((16, 8), dtype=torch.float64)), TypeError, "rays must be"),
        (dict(prim=torch.zeros(16, dtype=torch.int64)), TypeError, "prim must be"),
        (dict(t=torch.zeros(16, dtype=torch.float16)), TypeError, "t must be"),
        (dict(skip=torch.zeros(16, dtype=torch.float32)), TypeError, "skip must be"),
        (dict(prim=torch.zeros(15, dtype=torch.int32)), ValueError, "fewer than n"),
        (dict(t=torch.zeros(8)), ValueError, "fewer than n"),
        (dict(skip=torch.zeros(3, dtype=torch.int32)), ValueError, "fewer than n"),
        (dict(rays=torch.zeros((8, 16)).t()), ValueError, "contiguous"),
        ({}, ValueError, "CUDA tensor"),  # well-formed, but host memory
    ]
    for change, exc, text in cases:
        args = dict(ok, **change)
        with pytest.raises(exc, match=text):
            cr.check_static_trace_args(args["rays"], args["skip"], args["prim"], args["t"])
        with pytest.raises(exc, match=text):  # the entry point's wrapper checks before calling C
            cr.cr_trace_rays_static(None, args["rays"], args["skip"], args["prim"], args["t"])


def test_debug_sort_rejects_bad_arguments_without_gpu(cr):
    L = cr.lib()
    k = np.zeros(4, np.uint32)
    assert L.cr_debug_sort(None, None, 0, 1, None, None, None) == cr.CR_OK  # nothing to sort
    assert L.cr_debug_sort(k.ctypes.data, None, 4, 1, k.ctypes.data, k.ctypes.data, None) == cr.CR_ERR_INVALID_ARG
    assert L.cr_debug_sort(k.ctypes.data, k.ctypes.data, 4, 0, k.ctypes.data, k.ctypes.data, None) == \
        cr.CR_ERR_INVALID_ARG
