"""The library's lens model (csrc/lens.cuh: the SIE of Eqs. SIEX/SIEY plus
external shear, used by every ray-trace kernel) compiled for the host and
checked against the oracle's ray trace on many lenses: general SIEs, the
near-spherical switch to the SIS limit, strongly flattened lenses, shear,
rays at the exact lens centre and on the lens axes, and the bad-parameter
rule (finite, b >= 0, 0 < q <= 1)."""
import math
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle.lens import ray_trace

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lens_host(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("lens") / "lens_host")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-ffp-contract=off", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", "-I", os.path.join(HERE, "fft_host", "include"),
                        os.path.join(HERE, "fft_host", "lens_host.cpp"), "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host build failed: " + r.stderr[-400:])
    return exe


def _run(exe, cases):
    buf = [struct.pack("<i", len(cases))]
    for lens, x, y in cases:
        buf.append(np.asarray(lens, np.float64).tobytes())
        buf.append(struct.pack("<i", len(x)))
        buf.append(np.stack([x, y], axis=1).astype(np.float64).tobytes())
    r = subprocess.run([exe], input=b"".join(buf), capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    out, pos, res = r.stdout, 0, []
    for lens, x, _ in cases:
        bad = struct.unpack_from("<i", out, pos)[0]
        pos += 4
        b = np.frombuffer(out, dtype=np.float64, count=2 * len(x), offset=pos).reshape(-1, 2)
        pos += 16 * len(x)
        res.append((bad, b[:, 0], b[:, 1]))
    assert pos == len(out)
    return res


def test_ray_trace_matches_the_oracle(lens_host):
    rng = np.random.default_rng(7)
    g = np.linspace(-1.6, 1.6, 33)
    gx, gy = [a.ravel() for a in np.meshgrid(g, g)]
    cases = []
    for _ in range(200):
        lens = [rng.uniform(0.5, 1.5), rng.uniform(0.2, 1.0), rng.uniform(0, 2 * math.pi), rng.uniform(-0.2, 0.2),
                rng.uniform(-0.2, 0.2), rng.uniform(0, 0.15), rng.uniform(0, math.pi)]
        cases.append((lens, gx + rng.uniform(-0.01, 0.01), gy + rng.uniform(-0.01, 0.01)))
    for q in (1.0, 1.0 - 1e-7, 1.0 - 1e-5, 0.999, 0.05):   # SIS limit, its switch, strong flattening
        cases.append(([1.0, q, 0.7, 0.03, -0.02, 0.05, 1.0], gx, gy))
    # rays at the exact centre and on the lens axes
    x0, y0, phi = 0.1, -0.05, 0.3
    t = np.linspace(-1, 1, 21)
    ax = np.concatenate([[x0], x0 + t * math.cos(phi), x0 - t * math.sin(phi)])
    ay = np.concatenate([[y0], y0 + t * math.sin(phi), y0 + t * math.cos(phi)])
    cases.append(([1.0, 0.6, phi, x0, y0, 0.0, 0.0], ax, ay))
    res = _run(lens_host, cases)
    for (lens, x, y), (bad, bx, by) in zip(cases, res):
        assert bad == 0
        ox, oy = ray_trace(x, y, lens)
        np.testing.assert_allclose(bx, ox, atol=1e-12, err_msg=str(lens))
        np.testing.assert_allclose(by, oy, atol=1e-12, err_msg=str(lens))


def test_bad_parameters_are_flagged(lens_host):
    x = np.array([0.3])
    good = [1.0, 0.7, 0.5, 0.0, 0.0, 0.05, 1.0]
    bads = []
    for i, v in ((0, -0.1), (1, 0.0), (1, -0.5), (1, 1.0 + 1e-9), (0, float("nan")), (2, float("inf")),
                 (5, float("nan"))):
        lens = list(good)
        lens[i] = v
        bads.append((lens, x, x))
    res = _run(lens_host, [(good, x, x), ([0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0], x, x)] + bads)
    assert res[0][0] == 0 and res[1][0] == 0          # b = 0 and q = 1 are valid
    assert all(r[0] == 1 for r in res[2:])
