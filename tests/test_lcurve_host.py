"""The library's L-curve corner (csrc/lcurve.cuh, run by the finalize and
L-curve kernels) compiled for the host and checked against the oracle's
spline corner (oracle/lcurve.py, SciPy's natural CubicSpline) on thousands
of curves: L-curves of Tikhonov problems with random spectra, random
positive curves, and degenerate ones (fewer than three points, constant
values, merged duplicates, straight lines)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle.lcurve import lcurve_corner

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lcurve_host(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("lcurve") / "lcurve_host")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-ffp-contract=off", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", "-I", os.path.join(HERE, "fft_host", "include"),
                        os.path.join(HERE, "fft_host", "lcurve_host.cpp"), "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build failed: " + r.stderr[-400:])
    return exe


def _tikhonov_curve(rng, n):
    # chi2(lam) and ||s||^2(lam) of a Tikhonov problem with a random spectrum
    m = 60
    sv = np.exp(rng.uniform(-8, 0, m))
    beta = rng.standard_normal(m) * np.exp(rng.uniform(-3, 1, m))
    lams = np.logspace(rng.uniform(-7, -4), rng.uniform(0, 2), n)
    f = sv[None, :] ** 2 / (sv[None, :] ** 2 + lams[:, None])
    chi2 = ((1 - f) ** 2 * beta ** 2).sum(axis=1) + rng.uniform(1e-3, 1.0)
    reg = (f ** 2 * beta ** 2 / sv ** 2).sum(axis=1)
    return chi2, reg


def _curves(rng):
    out = []
    for _ in range(1500):
        out.append(_tikhonov_curve(rng, int(rng.integers(3, 65))))
    for _ in range(1000):
        n = int(rng.integers(1, 65))
        out.append((np.exp(rng.uniform(-5, 5, n)), np.exp(rng.uniform(-5, 5, n))))
    for n in range(0, 6):                                  # short and empty curves
        out.append((np.ones(n), np.ones(n)))
        out.append((np.arange(1, n + 1.0), np.arange(n + 1.0, 1, -1)))
    for _ in range(200):                                   # duplicated points merge
        chi2, reg = _tikhonov_curve(rng, 20)
        k = int(rng.integers(1, 19))
        chi2[k] = chi2[k - 1]
        reg[k] = reg[k - 1]
        out.append((chi2, reg))
    for _ in range(100):                                   # straight lines in log-log
        n = int(rng.integers(3, 40))
        a = rng.uniform(-2, 2)
        x = np.linspace(-3, 3, n)
        out.append((10.0 ** (a * x + 1), 10.0 ** x))
    return out


def test_corner_matches_the_oracle(lcurve_host):
    rng = np.random.default_rng(11)
    curves = _curves(rng)
    buf = [struct.pack("<i", len(curves))]
    for chi2, reg in curves:
        buf.append(struct.pack("<i", len(chi2)))
        buf.append(np.asarray(chi2, np.float64).tobytes())
        buf.append(np.asarray(reg, np.float64).tobytes())
    r = subprocess.run([lcurve_host], input=b"".join(buf), capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    out = r.stdout
    pos = 0
    moved = 0
    for i, (chi2, reg) in enumerate(curves):
        n = len(chi2)
        corner, flat = struct.unpack_from("<ii", out, pos)
        pos += 8
        kap = np.frombuffer(out, dtype=np.float64, count=n, offset=pos)
        pos += 8 * n
        c_o, k_o, f_o = lcurve_corner(chi2, reg)
        assert bool(flat) == f_o, (i, n, flat, f_o)
        np.testing.assert_allclose(kap, k_o, rtol=1e-7, atol=1e-9 * max(1.0, np.abs(k_o).max(initial=0.0)), err_msg=str(i))
        if corner != c_o:
            # only a near-tie of the curvature may move the corner
            assert abs(k_o[corner] - k_o[c_o]) <= 1e-6 * k_o[c_o], (i, corner, c_o)
            moved += 1
    assert pos == len(out)
    assert moved <= 3
