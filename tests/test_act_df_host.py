"""The FP64 path's softplus (csrc/act_df.cuh) evaluates z = log(1 + e^y), s = z' and
t = z'' in double-float arithmetic on the FP32 pipe. Its header compiles for the host
with the same FP32 operations, so the device arithmetic is swept here, on the CPU,
against extended-precision libm over the whole range: random pre-activations up to
|y| = 800 (the clamp at 700 included), both sides of every log-table cell, the edge of
the e < 2^-60 regime, and exact special values (y = 0, +-50)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sweep_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("actdf") / "act_df_sweep")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(HERE, "act_df_sweep.cpp"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def test_softplus_double_float_accuracy(sweep_exe):
    out = subprocess.run([sweep_exe, "1000000"], check=True, capture_output=True, text=True).stdout.split()
    zabs, srel, trel = (float(v) for v in out[:3])
    nonfinite, zero_ok, big_ok, small_ok = (int(v) for v in out[3:])
    # bounds of the arithmetic (float pairs carry about 2^-48 per operation; the swept
    # maxima are 7.0e-15, 2.0e-14 and 3.8e-14)
    assert zabs < 1.5e-14, zabs
    assert srel < 5e-14, srel
    assert trel < 8e-14, trel
    assert nonfinite == 0
    assert zero_ok and big_ok and small_ok
