"""The ray sort of the Morton comparator (TwoPoint and the other Table 1 keys, Sec. 4):
a stable LSD radix sort of 30-bit keys with their slots.  Integer work, so the check is
bit-exact against numpy's stable sort; CUB's radix sort on the same keys is a second,
independent cross-check and the timing reference."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cr():
    from paper_2310_07182_gb300 import binding
    binding.lib()
    return binding


def _expect(keys, vals):
    k = keys & np.uint32((1 << 30) - 1)
    order = np.argsort(k, kind="stable")
    return k[order], vals[order]


@pytest.mark.parametrize("n", [1, 2, 31, 511, 512, 4095, 4096, 4097, 12289, 100_003, 1_463_294, 2_073_600, 6_000_000])
def test_sort_matches_a_stable_sort(cr, n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)  # bits above 30 are ignored
    vals = rng.permutation(n).astype(np.int32)
    ko, vo, ms = cr.cr_debug_sort(keys, vals)
    ek, ev = _expect(keys, vals)
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)


@pytest.mark.parametrize("distinct", [1, 2, 7, 1024, 1025])
def test_sort_is_stable_under_heavy_duplication(cr, distinct):
    n = 300_000
    rng = np.random.default_rng(distinct)
    levels = rng.integers(0, 1 << 30, distinct, dtype=np.uint64).astype(np.uint32)
    keys = levels[rng.integers(0, distinct, n)]
    vals = np.arange(n, dtype=np.int32)
    ko, vo, _ = cr.cr_debug_sort(keys, vals)
    ek, ev = _expect(keys, vals)
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)


def test_sort_of_coherent_morton_like_keys_on_device(cr):
    """Keys that arrive nearly sorted in runs (as Morton codes of an image-ordered queue do),
    device tensors in and out."""
    n = 1_000_000
    rng = np.random.default_rng(5)
    base = np.repeat(rng.integers(0, 1 << 30, n // 64, dtype=np.int64), 64)[:n]
    keys = ((base + rng.integers(0, 4096, n, dtype=np.int64)) & ((1 << 30) - 1)).astype(np.uint32)
    vals = np.arange(n, dtype=np.int32)
    ko, vo, _ = cr.cr_debug_sort(torch.from_numpy(keys.view(np.int32)).cuda(), torch.from_numpy(vals).cuda())
    ek, ev = _expect(keys, vals)
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), ek) and np.array_equal(vo.cpu().numpy(), ev)


def test_cross_check_and_timing_against_cub(cr):
    src = os.path.join(HERE, "helpers", "cub_sort.cu")
    so = os.path.join(HERE, "helpers", "libcub_sort.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", so, src], check=True)
    lib = C.CDLL(so)
    for n in (550_000, 1_463_294):  # the landscape's bounce-2 and bounce-1 ray counts
        rng = np.random.default_rng(n)
        keys = torch.from_numpy(rng.integers(0, 1 << 30, n, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
        vals = torch.arange(n, dtype=torch.int32, device="cuda")
        ko, vo, ms = cr.cr_debug_sort(keys, vals, reps=20)
        kc, vc = torch.empty_like(keys), torch.empty_like(vals)
        ms_cub = C.c_float()
        assert lib.cub_sort_pairs(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), C.c_void_p(kc.data_ptr()),
                                  C.c_void_p(vc.data_ptr()), n, 30, 20, C.byref(ms_cub)) == 0
        assert torch.equal(ko, kc) and torch.equal(vo, vc)
        # algorithmic bytes: key kernel 4 + 4 in, 3 x 4 out; three passes of 8 in and 8 out
        gbs = n * (8 + 12 + 3 * 16) / (ms * 1e-3) / 1e9
        print(f"sort n={n}: {ms * 1e3:.1f} us ({gbs:.0f} GB/s algorithmic), CUB {ms_cub.value * 1e3:.1f} us")
