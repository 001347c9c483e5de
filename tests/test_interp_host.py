"""The bicubic weights the kernels use (csrc/interp.cuh: Keys' kernel
written out as cubics in the cell offset u) compiled for the host and
checked against the oracle's piecewise definition of the kernel."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.operators import keys_kernel

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bicubic_weights_match_the_oracle_kernel(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "keys_host")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-ffp-contract=off", "-I", os.path.join(HERE, "fft_host", "include"),
                        os.path.join(HERE, "fft_host", "keys_host.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-600:]
    n = 1001
    out = subprocess.run([exe, str(n)], capture_output=True, timeout=60)
    assert out.returncode == 0
    w = np.frombuffer(out.stdout, dtype=np.float64).reshape(n, 4)
    u = np.linspace(0.0, 1.0, n)
    ref = np.stack([keys_kernel(1 + u), keys_kernel(u), keys_kernel(1 - u), keys_kernel(2 - u)], axis=1)
    np.testing.assert_allclose(w, ref, atol=1e-15)
