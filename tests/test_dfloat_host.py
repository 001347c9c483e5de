"""The refinement's double-float accumulation (csrc/dfloat.cuh) compiled for
the host and checked against exact rational sums: sums of FP32 taps times
FP64 inputs, the shape of the refinement's convolutions, must carry about
2^-44 of relative error (against Sum |t x|), where an FP32 accumulation
carries ~2^-24 per term."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dfloat_host(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dfloat") / "dfloat_host")
    cmd = [gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", os.path.join(HERE, "fft_host", "include"),
           os.path.join(HERE, "fft_host", "dfloat_host.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build failed: " + r.stderr[-400:])
    return exe


@pytest.mark.parametrize("n,seed,signed", [(81, 0, False), (441, 1, False), (4225, 2, False), (81, 3, True),
                                           (441, 4, True)])
def test_double_float_sum_is_near_fp64(dfloat_host, n, seed, signed):
    rng = np.random.default_rng(seed)
    t = rng.random(n).astype(np.float32)          # a PSF: FP32 taps
    if signed:
        t = (t - 0.5).astype(np.float32)          # a general filter
    x = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))   # FP64 inputs over six decades
    r = subprocess.run([dfloat_host, str(n)], input=t.tobytes() + x.tobytes(), capture_output=True, timeout=60)
    assert r.returncode == 0
    s, c = np.frombuffer(r.stdout, dtype=np.float64)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(t, x))
    scale = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(t, x)))
    err = abs(float(Fraction(s) + Fraction(c) - exact)) / scale
    assert err <= 2.0 ** -40, err
    # the FP32 sum of the same products is far coarser: the pair is what
    # makes the FP32 pipe good enough for the refinement residual
    f32 = np.float32(0)
    for a, b in zip(t, x.astype(np.float32)):
        f32 = np.float32(f32 + a * b)
    assert abs(float(Fraction(float(f32)) - exact)) / scale > 100 * err
