"""Pins for the oracle's regularised solve and L-curve (Sections 2.1, 2.4, 2.6).

The solve is pinned by a closed form (identity lens, delta PSF, H = I), by
the SVD filter-factor expansion of Eq. tikFF, by noise-free recovery as
lambda -> 0 and by the normal-equation residual; the L-curve corner by
curves whose curvature is known.
"""
import math

import numpy as np
import pytest

import synth
from oracle.data import lensed_image, observe
from oracle.lcurve import lcurve_corner
from oracle.operators import REG_GRADIENT, REG_IDENTITY, REG_LAPLACIAN
from oracle.solve import (Problem, build_operators, chi2_of, eval_candidate, normal_residual_ld, reg_of,
                          solve_lambda, solve_lambda_refined)
from synth import Geometry, gaussian_psf

LENS = np.array([1.0, 0.7, 0.5, 0.0, 0.0, 0.05, 1.0])


def _small(reg=REG_GRADIENT, nsrc=8, seed=0):
    g = Geometry(nx=16, ny=16, pix=0.1, sx=nsrc, sy=nsrc, sxmin=-0.6, sxmax=0.6, symin=-0.6, symax=0.6,
                 kpsf=5, subpix=1, reg=reg)
    rng = np.random.default_rng(seed)
    return observe(g, LENS, synth.two_gaussian_source(), gaussian_psf(5, 1.0),
                   rng.standard_normal((16, 16)))


def test_closed_form_identity_lens():
    # L = I, B = I, H = I: (W + lam I) s = W d, s_j = w_j d_j / (w_j + lam)
    g = Geometry(nx=6, ny=5, pix=0.1, sx=6, sy=5, sxmin=-0.3, sxmax=0.3, symin=-0.25, symax=0.25,
                 kpsf=3, subpix=1, reg=REG_IDENTITY)
    rng = np.random.default_rng(1)
    psf = np.zeros((3, 3))
    psf[1, 1] = 1.0
    sig = rng.uniform(0.5, 2.0, (5, 6))
    mask = (rng.uniform(size=(5, 6)) > 0.2).astype(np.uint8)
    d = rng.standard_normal((5, 6))
    prob = Problem(g, d, sig, mask, psf)
    ops = build_operators(prob, [0.0, 0.8, 0.0, 0, 0, 0, 0])
    w = mask.ravel() / sig.ravel() ** 2
    for lam in (1e-3, 0.5, 10.0):
        s = solve_lambda(ops, lam)
        np.testing.assert_allclose(s, w * d.ravel() / (w + lam), rtol=1e-12, atol=1e-14)


def test_refined_solve_matches_exact_rational_solve():
    # the refined solve against the exact solution of the same normal
    # equations: A and rhs formed from the FP64 entries of L, B, W, H and d in
    # 60-digit arithmetic (mpmath) and solved there; an ill-conditioned case
    # (gradient H, lambda down to 1e-9)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    g = Geometry(nx=8, ny=8, pix=0.2, sx=4, sy=4, sxmin=-0.6, sxmax=0.6, symin=-0.6, symax=0.6,
                 kpsf=3, subpix=1, reg=REG_GRADIENT)
    rng = np.random.default_rng(3)
    prob = observe(g, LENS, synth.two_gaussian_source(), gaussian_psf(3, 1.0), rng.standard_normal((8, 8)))
    ops = build_operators(prob, LENS)
    M = lambda a: mpmath.matrix(np.asarray(a.toarray() if hasattr(a, "toarray") else a, dtype=np.float64).tolist())
    L, B, H = M(ops.L), M(ops.B), M(ops.H)
    W = mpmath.diag([mpmath.mpf(float(x)) for x in ops.w])
    d = mpmath.matrix([float(x) for x in np.asarray(prob.d, dtype=np.float64).ravel()])
    F = B * L
    FtW = F.T * W
    FtWF, HtH, rhs = FtW * F, H.T * H, FtW * d
    for lam in (1e-2, 1e-6, 1e-9):
        s_x = mpmath.lu_solve(FtWF + mpmath.mpf(lam) * HtH, rhs)
        s_x = np.array([float(v) for v in s_x])
        s_r = solve_lambda_refined(ops, prob, lam)
        assert np.linalg.norm(s_r - s_x) <= 4e-16 * np.linalg.norm(s_x) * np.sqrt(g.ns), lam
        r = np.asarray(normal_residual_ld(ops, prob, s_r, lam), dtype=np.float64)
        assert np.linalg.norm(r) <= 1e-15 * np.linalg.norm(ops.rhs), lam


def test_svd_filter_factors():
    # H = I: s = sum_i phi_i (u_i^T b / nu_i) v_i with phi_i = nu_i^2/(nu_i^2 + lam)  (Eq. tikFF)
    prob = _small(REG_IDENTITY)
    ops = build_operators(prob, LENS)
    Fh = np.sqrt(ops.w)[:, None] * ops.F
    bh = np.sqrt(ops.w) * prob.d.ravel()
    U, nu, Vt = np.linalg.svd(Fh, full_matrices=False)
    for lam in (1e-3, 1e-1, 10.0):
        phi = nu ** 2 / (nu ** 2 + lam)
        s_svd = Vt.T @ (phi * (U.T @ bh) / nu)
        np.testing.assert_allclose(solve_lambda(ops, lam), s_svd, rtol=1e-9, atol=1e-9 * np.abs(s_svd).max())


@pytest.mark.parametrize("reg", [REG_IDENTITY, REG_GRADIENT, REG_LAPLACIAN])
def test_normal_equation_residual(reg):
    prob = _small(reg)
    ops = build_operators(prob, LENS)
    for lam in (1e-4, 1e-2, 1.0, 1e2):
        s = solve_lambda(ops, lam)
        A = ops.FtWF + lam * ops.HtH
        assert np.linalg.norm(A @ s - ops.rhs) <= 1e-11 * np.linalg.norm(ops.rhs)


def test_noise_free_recovery():
    # d = B L s_true exactly; lam -> 0 recovers s_true where L has full column rank
    prob = _small(REG_GRADIENT, nsrc=6)
    ops = build_operators(prob, LENS)
    assert np.linalg.matrix_rank(ops.F[ops.w > 0]) == prob.geom.ns
    s_true = np.random.default_rng(5).uniform(0, 1, prob.geom.ns)
    prob2 = Problem(prob.geom, (ops.F @ s_true).reshape(16, 16), prob.sigma, prob.mask, prob.psf)
    ops2 = build_operators(prob2, LENS)
    s = solve_lambda(ops2, 1e-12)
    np.testing.assert_allclose(s, s_true, atol=1e-6)
    assert chi2_of(ops2, prob2.d, s) < 1e-12


def test_chi2_and_reg_definitions():
    prob = _small(REG_LAPLACIAN)
    ops = build_operators(prob, LENS)
    s = solve_lambda(ops, 0.1)
    # Eq. chi2 written out pixel by pixel
    model = ops.F @ s
    m = (prob.mask.ravel() != 0) & ops.mapped
    chi = sum((model[j] - prob.d.ravel()[j]) ** 2 / prob.sigma.ravel()[j] ** 2 for j in range(256) if m[j])
    assert abs(chi2_of(ops, prob.d, s) - chi) < 1e-10 * chi
    # Laplacian measure on the 2-D grid by hand
    S = s.reshape(8, 8)
    P = np.pad(S, 1)
    lap = 4 * S - P[:-2, 1:-1] - P[2:, 1:-1] - P[1:-1, :-2] - P[1:-1, 2:]
    assert abs(reg_of(ops, s) - float((lap ** 2).sum())) < 1e-10 * float((lap ** 2).sum())


def test_lcurve_monotone_tradeoff():
    # chi2 grows and ||Hs|| shrinks with lambda (Tikhonov trade-off)
    prob = _small(REG_LAPLACIAN)
    r = eval_candidate(prob, LENS, synth.lambda_grid(12))
    assert np.all(np.diff(r.chi2) > 0)
    assert np.all(np.diff(r.reg) < 0)
    assert 0 < r.corner < 11


def test_lcurve_circle():
    # points on a circle of radius R: kappa ~= 1/R at interior knots
    R = 2.5
    ang = np.linspace(0.2, 1.4, 25)
    x, y = R * np.cos(ang), R * np.sin(ang)
    corner, kappa, flat = lcurve_corner(10 ** y, 10 ** x)  # reg -> x axis, chi2 -> y axis
    assert not flat
    np.testing.assert_allclose(kappa[6:-6], 1.0 / R, rtol=5e-4)  # natural ends perturb ~5 knots
    assert kappa[0] == 0 and kappa[-1] == 0


def test_lcurve_symmetric_hyperbola():
    # y = 1/x sampled symmetrically about x = 1: the corner is the middle knot
    t = np.linspace(-1.5, 1.5, 15)
    x = np.exp(t)
    y = 1.0 / x
    corner, kappa, flat = lcurve_corner(10 ** y, 10 ** x)
    assert corner == 7 and not flat


def test_lcurve_straight_line_is_flat():
    x = np.linspace(0, 3, 9)
    corner, kappa, flat = lcurve_corner(10 ** (2 * x + 1), 10 ** x)
    assert flat and corner == 4


def test_lcurve_merges_duplicates():
    x = np.array([0.0, 0.5, 0.5, 1.0, 1.2, 1.3])
    y = np.array([3.0, 1.0, 1.0, 0.4, 0.3, 0.25])
    c1, k1, _ = lcurve_corner(10 ** y, 10 ** x)
    keep = [0, 1, 3, 4, 5]
    c2, k2, _ = lcurve_corner(10 ** y[keep], 10 ** x[keep])
    assert k1[2] == 0.0
    np.testing.assert_allclose(k1[keep], k2)


def test_observation_snr():
    g = synth.geom_small_fp64()
    rng = np.random.default_rng(0)
    prob = observe(g, LENS, synth.two_gaussian_source(), gaussian_psf(5, 1.0), rng.standard_normal((32, 32)))
    clean = lensed_image(g, LENS, synth.two_gaussian_source())
    from scipy.signal import convolve2d
    peak = convolve2d(clean, gaussian_psf(5, 1.0), mode="same").max()
    assert abs(prob.sigma[0, 0] - peak / 20.0) < 1e-15
