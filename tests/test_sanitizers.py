"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (compute-sanitizer is
not used): the oracle on a scene with every material type in every mode, and the host
BVH builders on random, heightfield and degenerate inputs.  Each helper is compiled with
-fsanitize=address,undefined -fno-sanitize-recover=all, so any report fails the run."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def _run(cmd_build, exe, tmp_path):
    if shutil.which(cmd_build[0]) is None:
        pytest.skip(f"{cmd_build[0]} not available")
    b = subprocess.run(cmd_build, capture_output=True, text=True)
    if b.returncode != 0:
        if "sanitize" in b.stderr and ("cannot find" in b.stderr or "unrecognized" in b.stderr):
            pytest.skip("sanitizer runtime not available")
        raise AssertionError(b.stderr[-3000:])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
    return r.stdout


def test_oracle_under_sanitizers(tmp_path):
    exe = str(tmp_path / "oracle_san")
    cmd = ["gcc", "-std=c11", "-ffp-contract=off", *SAN, "-I", os.path.join(ROOT, "oracle"),
           os.path.join(ROOT, "oracle", "oracle.c"), os.path.join(HERE, "helpers", "oracle_sanitize_main.c"),
           "-o", exe, "-lm", "-lpthread"]
    assert "oracle sanitize run ok" in _run(cmd, exe, tmp_path)


def test_bvh_builders_under_sanitizers(tmp_path):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path / "bvh_san")
    csrc = os.path.join(ROOT, "paper_2310_07182_gb300", "csrc")
    cmd = ["g++", "-std=c++17", *SAN, "-I", os.path.join(ROOT, "include"), "-I", csrc, "-I", inc,
           os.path.join(csrc, "bvh_build.cpp"), os.path.join(csrc, "bvh8_build.cpp"),
           os.path.join(HERE, "helpers", "bvh_sanitize_main.cpp"),
           "-o", exe, "-lpthread"]
    assert "bvh sanitize run ok" in _run(cmd, exe, tmp_path)
