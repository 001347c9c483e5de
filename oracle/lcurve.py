"""Oracle: L-curve corner by maximum curvature (Section 2.6), FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The L-curve points are (x_k, y_k) = (log10 R_k, log10 chi2_k) in lambda
order, R_k = ||H s_k||^2 the regularisation measure and chi2_k the image
chi^2.  Following Section 2.6 the curve is parameterised by arclength (here
the cumulative chord length t between the points), x(t) and y(t) are each
fitted with a cubic spline (natural end conditions), and the curvature

    kappa = |x' y'' - y' x''| / (x'^2 + y'^2)^(3/2)

is evaluated at the knots; the corner is the knot of maximum kappa (ties go
to the smaller lambda index).  The natural end conditions make kappa zero at
the two end knots, which are never chosen.  Points closer than 1e-12 of the total chord
length to their predecessor are merged into it (kappa 0).  With fewer than
three distinct points, or kappa times the total chord length at most 1e-9
everywhere (a straight line up to rounding), the middle index is returned
and the curve is flagged flat.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import CubicSpline

TINY = 1e-300
MERGE_REL = 1e-12
# kappa * total chord length at or below this counts as a straight line
FLAT_REL = 1e-9


def lcurve_points(chi2, reg):
    """(x, y) = (log10 R, log10 chi2), values floored at 1e-300."""
    x = np.log10(np.maximum(np.asarray(reg, dtype=np.float64), TINY))
    y = np.log10(np.maximum(np.asarray(chi2, dtype=np.float64), TINY))
    return x, y


def lcurve_corner(chi2, reg):
    """Return (corner index, kappa[n], flat flag)."""
    x, y = lcurve_points(chi2, reg)
    n = len(x)
    kappa = np.zeros(n)
    if n < 3:
        return (n - 1) // 2 if n > 0 else 0, kappa, True
    step = np.hypot(np.diff(x), np.diff(y))
    total = float(step.sum())
    keep = np.ones(n, dtype=bool)
    if total > 0:
        keep[1:] = step > MERGE_REL * total
    else:
        keep[1:] = False
    idx = np.flatnonzero(keep)
    if len(idx) < 3:
        return (n - 1) // 2, kappa, True
    xs, ys = x[idx], y[idx]
    t = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(xs), np.diff(ys)))])
    sx = CubicSpline(t, xs, bc_type="natural")
    sy = CubicSpline(t, ys, bc_type="natural")
    x1, x2 = sx(t, 1), sx(t, 2)
    y1, y2 = sy(t, 1), sy(t, 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.abs(x1 * y2 - y1 * x2) / np.power(x1 * x1 + y1 * y1, 1.5)
    # a knot where the spline's tangent vanishes has no defined curvature
    k = np.where(np.isfinite(k), k, 0.0)
    # natural end conditions: the second derivatives vanish at the end knots
    k[0] = 0.0
    k[-1] = 0.0
    kappa[idx] = k
    if not np.any(kappa * t[-1] > FLAT_REL):
        return (n - 1) // 2, kappa, True
    return int(np.argmax(kappa)), kappa, False
