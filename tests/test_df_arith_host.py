"""The complex128 double-float arithmetic of the kernels (packed f32x2 lanes, the tile-pass
phase frame), built for the host and checked against long double.

Bounds: one double-float operation keeps ~2^-45 of the operand magnitudes (TwoProduct and
TwoSum are exact; the first-order cross terms and the final low-part sums are rounded in
binary32, ~2^-24 of a term that is itself ~2^-22 of the result); the split of a binary64
into hi + lo keeps 2^-47.  A chain of 64 rotation + phase steps stays within 64 times the
one-step bound.  rot_q (multiplication by a power of -i) is exact.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def df_errors(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("df") / "df_arith_host")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
           "-o", out, os.path.join(HERE, "df_arith_host.cu"),
           os.path.join(ROOT, "paper_2010_09746_gb300", "csrc", "gates.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return {k: float(v) for k, v in (line.split() for line in r.stdout.strip().splitlines())}


def test_split_join_round_trip(df_errors):
    assert df_errors["roundtrip"] <= 2.0 ** -46


@pytest.mark.parametrize("name", ["mul", "rx", "axpy", "axmy", "ymx", "rot"])
def test_one_operation(df_errors, name):
    assert df_errors[name] <= 2.0 ** -43, (name, df_errors[name])


def test_frame_rotation_exact(df_errors):
    assert df_errors["rot_q"] == 0.0


def test_chain_of_64_steps(df_errors):
    assert df_errors["chain64"] <= 64 * 2.0 ** -43, df_errors["chain64"]
