"""The library's regulariser (csrc/reg.cuh: H v, H^T r and diag(H^T H) of
Eq. TKReg with H = I, the forward-difference gradient or the 5-point
Laplacian, zero beyond the grid) compiled for the host and checked against
the oracle's explicit H on square and ragged grids."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.operators import reg_matrix

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def reg_host(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("reg") / "reg_host")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-I",
                        os.path.join(HERE, "fft_host", "include"), os.path.join(HERE, "fft_host", "reg_host.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build failed: " + r.stderr[-400:])
    return exe


@pytest.mark.parametrize("reg", [synth.REG_IDENTITY, synth.REG_GRADIENT, synth.REG_LAPLACIAN])
@pytest.mark.parametrize("sx,sy", [(1, 1), (2, 3), (7, 5), (16, 16), (13, 24)])
def test_regulariser_matches_the_oracle(reg_host, reg, sx, sy):
    g = synth.Geometry(8, 8, 0.1, sx, sy, -0.8, 0.8, -0.8, 0.8, 3, 1, reg)
    H = reg_matrix(g, reg).toarray()
    rng = np.random.default_rng(sx * 100 + sy * 10 + reg)
    v = rng.standard_normal(H.shape[1])
    r = rng.standard_normal(H.shape[0])
    out = subprocess.run([reg_host, str(sx), str(sy), str(reg)], input=v.tobytes() + r.tobytes(),
                         capture_output=True, timeout=60)
    assert out.returncode == 0, out.stderr.decode()[-1000:]
    a = np.frombuffer(out.stdout, dtype=np.float64)
    nreg, ns = H.shape
    hv, htr, d = a[:nreg], a[nreg:nreg + ns], a[nreg + ns:]
    np.testing.assert_allclose(hv, H @ v, atol=1e-13)
    np.testing.assert_allclose(htr, H.T @ r, atol=1e-13)
    np.testing.assert_allclose(d, np.diag(H.T @ H), atol=0)
