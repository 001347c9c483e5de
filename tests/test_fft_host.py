"""The library's FFT convolution (csrc/fftconv.cuh) compiled for the host
and checked against the oracle's explicit blur matrix.

The CUDA source runs unchanged as one thread (tests/fft_host/include
supplies stand-ins for the CUDA names); AddressSanitizer turns any index
outside the buffers the kernel carves (twiddle tables, batch buffers, half
spectra) into a failure.  The cases cover every grid side from 16 to 1024,
odd and ragged image sizes, PSFs wider than the image and than the grid,
FP32 and FP64, B and B^T.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.operators import blur_matrix

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fft_host(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("fft_host") / "fft_host")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-I", os.path.join(HERE, "fft_host", "include"),
           os.path.join(HERE, "fft_host", "fft_host.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build of the FFT harness failed: " + r.stderr[-400:])
    return exe


def _run(exe, img, psf, prec, corr):
    ny, nx = img.shape
    k = psf.shape[0]
    data = np.ascontiguousarray(img, dtype=np.float64).tobytes() + np.ascontiguousarray(psf, np.float64).tobytes()
    r = subprocess.run([exe, str(nx), str(ny), str(k), str(prec), str(int(corr))], input=data,
                       capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    m = int(r.stderr.decode().strip().split("M=")[-1])
    return np.frombuffer(r.stdout, dtype=np.float64).reshape(ny, nx), m


@pytest.mark.parametrize("ny,nx,k,expect_m", [
    (7, 5, 3, 16),        # smallest grid
    (13, 11, 9, 32),
    (40, 36, 65, 128),    # PSF wider than the image
    (9, 6, 41, 32),       # PSF wider than the grid: taps share grid points
    (64, 64, 9, 128),
    (150, 97, 21, 256),
    (480, 300, 5, 512),
    (1000, 37, 3, 1024),
])
@pytest.mark.parametrize("prec", [32, 64])
def test_fft_convolution_matches_the_blur_matrix(fft_host, ny, nx, k, expect_m, prec):
    rng = np.random.default_rng(ny * 1000 + nx + k)
    img = rng.standard_normal((ny, nx))
    psf = rng.random((k, k))
    g = synth.Geometry(nx, ny, 0.1, 4, 4, -0.8, 0.8, -0.8, 0.8, k, 1, synth.REG_IDENTITY)
    B = blur_matrix(g, psf, dense=False)
    for corr in (False, True):
        ref = (B.T if corr else B) @ img.ravel()
        got, m = _run(fft_host, img, psf, prec, corr)
        assert m == expect_m
        scale = np.abs(psf).sum() * np.abs(img).max()
        # FP32: log2(M^2) radix-2 stages each adding ~u relative error
        tol = (4 * 2 * np.log2(m) * 2.0 ** -24) if prec == 32 else 1e-13
        err = np.abs(got.ravel() - ref).max() / scale
        assert err <= tol, (corr, err, tol)
