"""Pins taken from values the paper prints (tests/golden/).

Section 4.2's Table 1 of optimiser results for the SIE example: both
optimisers return an orientation of 4.713 rad for a true pi/2 while matching
the data (reduced chi^2 1.010 and 1.012 against the true lens's 0.998).
That is only possible if the SIE's deflection field is pi-periodic in its
orientation, as the oracle's lens model has it: the field at 4.713 must
match the field at pi/2 up to the small angle 4.713 - 3 pi / 2.
"""
import math
import os

import numpy as np

from oracle.lens import deflection

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sie_orientation_table.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        rows[name] = [float(v) for v in vals]
    return rows


def test_recovered_orientation_is_the_true_one_modulo_pi():
    t = _table()
    ferret, locust, true = t["theta_L"]
    q = 1.0 - t["epsilon"][2]                        # the true ellipticity as an axis ratio
    g = np.linspace(-1.5, 1.5, 41)
    tx, ty = [a.ravel() for a in np.meshgrid(g, g)]
    ax_t, ay_t = deflection(tx, ty, [1.0, q, true, 0.0, 0.12, 0.0, 0.0])
    for found in (ferret, locust):
        ax_f, ay_f = deflection(tx, ty, [1.0, q, found, 0.0, 0.12, 0.0, 0.0])
        # the field turned by pi is the same field
        ax_p, ay_p = deflection(tx, ty, [1.0, q, found - math.pi, 0.0, 0.12, 0.0, 0.0])
        np.testing.assert_allclose(ax_f, ax_p, atol=1e-12)
        np.testing.assert_allclose(ay_f, ay_p, atol=1e-12)
        # and the recovered orientation reproduces the true field to the
        # first order of its offset from 3 pi / 2 (rotating by d moves the
        # deflection by at most ~2 b (1 - q) d for this ellipticity)
        d = abs(found - 1.5 * math.pi)
        assert d < 1e-3
        dev = np.hypot(ax_f - ax_t, ay_f - ay_t).max()
        assert dev <= 4.0 * (1.0 - q) * d + 1e-12, (dev, d)
        # whereas a quarter turn away the fields differ at order (1 - q)
        ax_q, ay_q = deflection(tx, ty, [1.0, q, true + 0.5 * math.pi, 0.0, 0.12, 0.0, 0.0])
        assert np.hypot(ax_q - ax_t, ay_q - ay_t).max() > 0.05
