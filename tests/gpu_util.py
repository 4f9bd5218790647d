"""Shared helpers of the GPU parity tests."""
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def radiance_close(got, ref, ok=None, rtol=1e-4, floor=1e-2):
    """|got - ref| <= rtol * max(|ref|, floor) per channel (relative 1e-4, and 1e-6 absolute
    below 1e-2), over the pixels selected by ``ok``.  Returns (all_close, max_excess, n_bad)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tol = rtol * np.maximum(np.abs(ref), floor)
    bad = np.abs(got - ref) > tol
    if ok is not None:
        bad &= ok[..., None] if ok.ndim == got.ndim - 1 else ok
    return (not bad.any()), float((np.abs(got - ref) - tol).max()), int(bad.any(axis=-1).sum())


def build_curand_helper():
    src = os.path.join(HERE, "helpers", "curand_philox.cu")
    out = os.path.join(HERE, "helpers", "libcurand_philox.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", out, src], check=True)
    return out
