"""The library's FFT convolution (csrc/fftconv.cuh) run by many host threads
as one CTA (per-thread threadIdx, __syncthreads() as a barrier) under
ThreadSanitizer: no two threads may touch the same element between
barriers with one of them writing, and B and B^T must still match the
oracle's blur matrix.  The sizes put several batches through every pass
and leave ragged last batches; the thread counts include ones that do not
divide the batch sizes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.operators import blur_matrix

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fft_mt(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("fft_mt") / "fft_host_mt")
    r = subprocess.run([gxx, "-std=c++20", "-O1", "-g", "-fsanitize=thread", "-I",
                        os.path.join(HERE, "fft_host", "include_mt"), os.path.join(HERE, "fft_host", "fft_host_mt.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build with ThreadSanitizer failed: " + r.stderr[-400:])
    probe = subprocess.run([exe, "4", "4", "3", "2"], input=np.zeros(25).tobytes(), capture_output=True, timeout=120)
    if probe.returncode != 0 and b"ThreadSanitizer" in probe.stderr and b"data race" not in probe.stderr:
        pytest.skip("ThreadSanitizer cannot run here: " + probe.stderr.decode()[-300:])
    return exe


@pytest.mark.parametrize("ny,nx,k,nt", [(40, 37, 9, 32), (13, 11, 9, 7), (70, 60, 21, 64), (9, 6, 41, 24)])
def test_fft_convolution_is_race_free_and_exact(fft_mt, ny, nx, k, nt):
    rng = np.random.default_rng(ny + nx + k + nt)
    img = rng.standard_normal((ny, nx))
    psf = rng.random((k, k))
    r = subprocess.run([fft_mt, str(nx), str(ny), str(k), str(nt)], input=img.tobytes() + psf.tobytes(),
                       capture_output=True, timeout=600)
    err = r.stderr.decode()
    assert "ThreadSanitizer" not in err, err[-3000:]
    assert r.returncode == 0, err[-2000:]
    out = np.frombuffer(r.stdout, dtype=np.float64)
    g = synth.Geometry(nx, ny, 0.1, 4, 4, -0.8, 0.8, -0.8, 0.8, k, 1, synth.REG_IDENTITY)
    B = blur_matrix(g, psf, dense=False)
    scale = np.abs(psf).sum() * np.abs(img).max()
    m = max(16, 1 << int(np.ceil(np.log2(max(nx, ny) + (k - 1) // 2))))
    tol = 8 * np.log2(m) * 2.0 ** -24
    assert np.abs(out[:ny * nx] - B @ img.ravel()).max() / scale <= tol
    assert np.abs(out[ny * nx:] - B.T @ img.ravel()).max() / scale <= tol
