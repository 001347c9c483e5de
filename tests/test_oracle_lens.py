"""Pins for the oracle's ray tracing (Eqs. thinlens, SIEX, SIEY).

Each test checks the oracle against something other than itself: the
spherical closed form, an independent numerical integral of the SIE
convergence, the Poisson equation and curl-freeness of a deflection field,
linearity of the shear, and the Einstein ring of an aligned source.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.lens import deflection, ray_trace, sie_alpha


def test_sis_closed_form():
    # q -> 1: alpha = b theta / |theta| (singular isothermal sphere)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-2, 2, 50), rng.uniform(-2, 2, 50)
    b = 1.3
    r = np.hypot(x, y)
    ax, ay = sie_alpha(x, y, b, 1.0)
    np.testing.assert_allclose(ax, b * x / r, rtol=1e-14)
    np.testing.assert_allclose(ay, b * y / r, rtol=1e-14)
    # the elliptical branch approaches the same limit
    ax2, ay2 = sie_alpha(x, y, b, 1.0 - 2e-6)
    np.testing.assert_allclose(ax2, b * x / r, atol=5e-6)
    np.testing.assert_allclose(ay2, b * y / r, atol=5e-6)


def _homoeoid_alpha(x, y, b, q):
    """Deflection of kappa = b / (2 xi), xi^2 = x^2 + y^2/q^2, by the
    homoeoid integrals alpha_x = q x J0, alpha_y = q y J1 (Schramm 1990),
    J_n = int_0^1 kappa(xi(u)) / (1 - (1-q^2) u)^(n+1/2) du with
    xi(u)^2 = u (x^2 + y^2 / (1 - (1-q^2) u))."""
    e2 = 1.0 - q * q

    def kap(u):
        xi = math.sqrt(u * (x * x + y * y / (1.0 - e2 * u)))
        return b / (2.0 * xi)

    j0 = quad(lambda u: kap(u) / (1.0 - e2 * u) ** 0.5, 0, 1, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    j1 = quad(lambda u: kap(u) / (1.0 - e2 * u) ** 1.5, 0, 1, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    return q * x * j0, q * y * j1


@pytest.mark.parametrize("q", [0.5, 0.7, 0.9])
def test_sie_against_convergence_integral(q):
    rng = np.random.default_rng(1)
    b = 1.1
    for _ in range(6):
        x, y = rng.uniform(-1.5, 1.5, 2)
        ax, ay = sie_alpha(np.array([x]), np.array([y]), b, q)
        hx, hy = _homoeoid_alpha(x, y, b, q)
        assert abs(ax[0] - hx) < 1e-9 * max(1.0, abs(hx))
        assert abs(ay[0] - hy) < 1e-9 * max(1.0, abs(hy))


def test_sie_poisson_and_curl():
    # (1/2) div alpha = kappa = b q / (2 psi) and curl alpha = 0
    b, q, h = 1.0, 0.6, 1e-5
    for x, y in [(0.3, 0.7), (-0.9, 0.2), (0.5, -0.5)]:
        axp, _ = sie_alpha(np.array([x + h]), np.array([y]), b, q)
        axm, _ = sie_alpha(np.array([x - h]), np.array([y]), b, q)
        _, ayp = sie_alpha(np.array([x]), np.array([y + h]), b, q)
        _, aym = sie_alpha(np.array([x]), np.array([y - h]), b, q)
        div = (axp - axm) / (2 * h) + (ayp - aym) / (2 * h)
        psi = math.sqrt(q * q * x * x + y * y)
        assert abs(0.5 * div[0] - b * q / (2 * psi)) < 1e-6
        _, ayxp = sie_alpha(np.array([x + h]), np.array([y]), b, q)
        _, ayxm = sie_alpha(np.array([x - h]), np.array([y]), b, q)
        axyp, _ = sie_alpha(np.array([x]), np.array([y + h]), b, q)
        axym, _ = sie_alpha(np.array([x]), np.array([y - h]), b, q)
        curl = (ayxp - ayxm) / (2 * h) - (axyp - axym) / (2 * h)
        assert abs(curl[0]) < 1e-6


def test_rotation_and_centre():
    # rotating the lens by phi rotates its deflection field with it
    rng = np.random.default_rng(2)
    x, y = rng.uniform(-1, 1, 20), rng.uniform(-1, 1, 20)
    b, q, phi = 1.0, 0.6, 0.8
    c, s = math.cos(phi), math.sin(phi)
    # points given in the lens frame, mapped to the sky by R(phi)
    xs, ys = c * x - s * y, s * x + c * y
    ax0, ay0 = sie_alpha(x, y, b, q)
    ax, ay = deflection(xs + 0.2, ys - 0.1, [b, q, phi, 0.2, -0.1, 0.0, 0.0])
    np.testing.assert_allclose(ax, c * ax0 - s * ay0, atol=1e-13)
    np.testing.assert_allclose(ay, s * ax0 + c * ay0, atol=1e-13)


def test_pi_periodicity():
    # an ellipse rotated by pi is the same ellipse
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, 1, 20), rng.uniform(-1, 1, 20)
    l1 = [1.2, 0.7, 0.4, 0.05, -0.03, 0.04, 0.3]
    l2 = list(l1)
    l2[2] += math.pi
    l2[6] += math.pi
    a1 = deflection(x, y, l1)
    a2 = deflection(x, y, l2)
    np.testing.assert_allclose(a1[0], a2[0], atol=1e-12)
    np.testing.assert_allclose(a1[1], a2[1], atol=1e-12)


def test_shear_is_linear_and_traceless():
    # pure shear (b = 0): alpha = [[g1, g2], [g2, -g1]] (theta - centre)
    gam, thg, x0, y0 = 0.07, 0.6, 0.1, -0.2
    g1, g2 = gam * math.cos(2 * thg), gam * math.sin(2 * thg)
    x, y = np.array([0.3, -0.4, 1.0]), np.array([0.2, 0.9, -1.1])
    ax, ay = deflection(x, y, [0.0, 0.8, 0.3, x0, y0, gam, thg])
    np.testing.assert_allclose(ax, g1 * (x - x0) + g2 * (y - y0), atol=1e-15)
    np.testing.assert_allclose(ay, g2 * (x - x0) - g1 * (y - y0), atol=1e-15)


def test_einstein_ring():
    # An SIS and a source on the optical axis: every ray at |theta| = b maps
    # to beta = 0, and radial rays map to |beta| = | |theta| - b |.
    b = 1.0
    ang = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    for r in (0.5, 1.0, 1.7):
        bx, by = ray_trace(r * np.cos(ang), r * np.sin(ang), [b, 1.0, 0.0, 0, 0, 0, 0])
        np.testing.assert_allclose(np.hypot(bx, by), abs(r - b), atol=1e-14)


def test_centre_ray_is_not_deflected():
    ax, ay = sie_alpha(np.array([0.0]), np.array([0.0]), 1.0, 0.7)
    assert ax[0] == 0.0 and ay[0] == 0.0
