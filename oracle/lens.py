"""Oracle: thin-lens ray tracing through an SIE plus external shear (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* Eq. thinlens (Section 2): beta = theta - alpha(theta).
* Eqs. SIEX / SIEY (Section 2.3): SIE deflection in the lens frame with core
  s = 0 (the paper keeps s fixed at zero), psi^2 = q^2 x^2 + y^2.
* Orientation: lens-frame coordinates are the image coordinates shifted by
  the lens centre and rotated by -phi; the deflection is rotated back by phi.
* External shear (not in the paper): gamma1 = gamma cos 2 theta_g,
  gamma2 = gamma sin 2 theta_g, alpha_g = (g1 x + g2 y, g2 x - g1 y) about
  the lens centre.
"""
from __future__ import annotations

import numpy as np

# Axis ratios this close to 1 use the spherical limit (alpha = b theta/|theta|).
Q_SPHERICAL = 1.0 - 1e-6


def sie_alpha(x: np.ndarray, y: np.ndarray, b: float, q: float):
    """Lens-frame SIE deflection, Eqs. SIEX/SIEY with s = 0.

    Returns (alpha_x, alpha_y).  At the centre (psi = 0) the deflection is
    taken as zero.  For q within 1e-6 of 1 the singular isothermal sphere
    form b (x, y)/r is used (the q -> 1 limit of the same equations).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ax = np.zeros(np.broadcast(x, y).shape)
    ay = np.zeros_like(ax)
    if q >= Q_SPHERICAL:
        r = np.hypot(x, y)
        nz = r > 0
        ax[nz] = b * (x * np.ones_like(ax))[nz] / r[nz]
        ay[nz] = b * (y * np.ones_like(ax))[nz] / r[nz]
        return ax, ay
    psi = np.sqrt(q * q * x * x + y * y)
    f = np.sqrt(1.0 - q * q)
    nz = psi > 0
    xb = (x * np.ones_like(ax))[nz]
    yb = (y * np.ones_like(ax))[nz]
    ax[nz] = b * q / f * np.arctan(xb * f / psi[nz])
    ay[nz] = b * q / f * np.arctanh(yb * f / psi[nz])
    return ax, ay


def deflection(tx: np.ndarray, ty: np.ndarray, lens):
    """Total deflection (SIE rotated by phi plus external shear) at image points.

    ``lens`` = (b, q, phi, x0, y0, gamma, theta_g).
    """
    b, q, phi, x0, y0, gam, thg = [float(v) for v in lens]
    dx = np.asarray(tx, dtype=np.float64) - x0
    dy = np.asarray(ty, dtype=np.float64) - y0
    c, s = np.cos(phi), np.sin(phi)
    xl = c * dx + s * dy
    yl = -s * dx + c * dy
    axl, ayl = sie_alpha(xl, yl, b, q)
    ax = c * axl - s * ayl
    ay = s * axl + c * ayl
    g1, g2 = gam * np.cos(2.0 * thg), gam * np.sin(2.0 * thg)
    ax = ax + g1 * dx + g2 * dy
    ay = ay + g2 * dx - g1 * dy
    return ax, ay


def ray_trace(tx: np.ndarray, ty: np.ndarray, lens):
    """Eq. thinlens: source-plane positions beta = theta - alpha(theta)."""
    ax, ay = deflection(tx, ty, lens)
    return np.asarray(tx, dtype=np.float64) - ax, np.asarray(ty, dtype=np.float64) - ay
