"""GPU parity for PSFs wider than the compiled tap sizes (up to the 65 x 65
class of the paper's large test, Section 2.7), against the FP64 oracle.

Such PSFs run on the runtime-K kernels (and, for the lambda grid in FP32
contexts, on the FFT convolution when it is selected).  The gates are the
bilinear tests' gates.  The images are small so that the dense oracle stays
fast; a 65 x 65 PSF on a 40 x 36 image spreads every pixel over the whole
image, which exercises every tap.
"""
import numpy as np
import pytest
import torch

import synth
from oracle.iterlc import cgls_iterations
from oracle.lcurve import lcurve_corner
from oracle.solve import eval_candidate, forward_chi2
from synth import Geometry, REG_GRADIENT, REG_LAPLACIAN

from .helpers import device_problem, make_problem
from .test_gpu_parity import _fp32_checks, _lam_t, _lens_t, ctx32, ctx64, mods  # noqa: F401 (fixtures)

pytestmark = pytest.mark.gpu

LENS = [1.05, 0.65, 0.3, 0.03, -0.02, 0.04, 0.7]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("geom", [
    Geometry(40, 36, 0.08, 20, 18, -0.8, 0.8, -0.7, 0.7, 65, 1, REG_LAPLACIAN),
    Geometry(48, 48, 0.07, 24, 24, -0.8, 0.8, -0.8, 0.8, 33, 2, REG_GRADIENT),
])
def test_forward_wide_psf(mods, ctx32, ctx64, precision, geom):
    ctx = ctx32 if precision == "fp32" else ctx64
    dt = torch.float32 if precision == "fp32" else torch.float64
    prob = make_problem(geom, seed=17, psf_sigma=geom.kpsf / 6.0)
    S = np.random.default_rng(18).uniform(0, 1, (4, geom.ns))
    m_o, c_o = forward_chi2(prob, LENS, S)
    m_g, c_g, st = ctx.forward(device_problem(prob, dt), _lens_t(LENS)[0], torch.as_tensor(S, dtype=dt, device="cuda"))
    # FP32: each model pixel is a sum of K^2 products, whose rounding error
    # grows like sqrt(K^2) u (u = 2^-24): the 2e-6 gate of the narrow PSFs,
    # or 4 K u for the wide ones
    tol = max(2e-6, 4 * geom.kpsf * 2.0 ** -24) if precision == "fp32" else 1e-12
    assert int(st.item()) == 0
    m_g = m_g.double().cpu().numpy()
    assert np.abs(m_g - m_o).max() <= tol * np.abs(m_o).max()
    np.testing.assert_allclose(c_g.cpu().numpy(), c_o, rtol=50 * tol)


@pytest.mark.parametrize("variant", [6, 5])
def test_eval_fp32_wide_psf(mods, ctx32, variant):
    # 48x48 image, 24x24 source, 33x33 PSF (sigma 5.5 px): direct runtime-K
    # convolution (variant 6) and the FFT convolution (variant 5)
    g = Geometry(48, 48, 0.07, 24, 24, -0.8, 0.8, -0.8, 0.8, 33, 1, REG_LAPLACIAN)
    prob = make_problem(g, seed=19, psf_sigma=5.5)
    lams = synth.lambda_grid(8, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS, [1.1, 0.6, 2.0, -0.05, 0.04, 0.08, 2.5]]
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0, 0], _lam_t(lams, 2), [8, 8], tol=1e-6,
                           want_all_x=True, variant=variant)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


@pytest.mark.parametrize("variant", [6, 0])
def test_eval_fp32_65px_psf(mods, ctx32, variant):
    # direct (variant 6) and the automatic choice (FFT at this width)
    g = Geometry(40, 36, 0.08, 20, 18, -0.8, 0.8, -0.7, 0.7, 65, 1, REG_LAPLACIAN)
    prob = make_problem(g, seed=23, psf_sigma=6.0)
    lams = synth.lambda_grid(6, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS]
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0], _lam_t(lams, 1), [6], tol=1e-6,
                           want_all_x=True, variant=variant)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


@pytest.mark.parametrize("variant", [6, 0])
def test_eval_fp64_65px_psf(mods, ctx64, variant):
    g = Geometry(32, 32, 0.1, 16, 16, -0.8, 0.8, -0.8, 0.8, 65, 1, REG_GRADIENT)
    prob = make_problem(g, seed=29, psf_sigma=4.0)
    lams = synth.lambda_grid(6, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS, [0.95, 0.75, 0.4, 0.02, -0.03, 0.03, 0.8]]
    out = ctx64.eval_batch([device_problem(prob, torch.float64)], _lens_t(lenses), [0, 0], _lam_t(lams, 2),
                           [6, 6], tol=1e-12, maxit=50000, variant=variant)
    for c, lens in enumerate(lenses):
        r = eval_candidate(prob, lens, lams)
        np.testing.assert_allclose(out["chi2"][c].cpu().numpy(), r.chi2, rtol=1e-9)
        assert int(out["corner"][c].item()) == r.corner


def test_iter_lcurve_65px_psf(mods, ctx64):
    g = Geometry(32, 32, 0.1, 16, 16, -0.8, 0.8, -0.8, 0.8, 65, 1, REG_GRADIENT)
    prob = make_problem(g, seed=31, psf_sigma=4.0)
    rng = np.random.default_rng(3)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 1)])
    out = ctx64.eval_iter([device_problem(prob, torch.float64)], _lens_t(lenses), [0, 0], 20)
    for c, lens in enumerate(lenses):
        r = cgls_iterations(prob, lens, 20)
        chi = out["chi2"][c].cpu().numpy()
        assert np.all(np.abs(chi[:7] / r.chi2[:7] - 1) <= 1e-12), (c, chi[:7], r.chi2[:7])
        cn = lcurve_corner(chi[1:], out["reg"][c].cpu().numpy()[1:])[0] + 1
        assert int(out["corner"][c]) == cn


def test_psf_wider_than_the_limit_is_rejected(mods, ctx32):
    g = Geometry(40, 36, 0.08, 20, 18, -0.8, 0.8, -0.7, 0.7, 67, 1, REG_LAPLACIAN)
    from oracle.solve import Problem
    prob = Problem(g, np.zeros((36, 40)), np.ones((36, 40)), np.ones((36, 40), np.uint8), np.ones((67, 67)) / 67 ** 2)
    with pytest.raises(Exception):
        ctx32.forward(device_problem(prob), _lens_t(LENS)[0], torch.zeros((1, g.ns), device="cuda"))


# ---------------------------------------------------------------------------
# the FFT convolution forced (variant 5) on the standard systems
# ---------------------------------------------------------------------------
def test_eval_fp32_fft_forced_64px(mods, ctx32):
    # the 64x64 GA system (9x9 PSF) with both convolutions of every CG
    # iteration and of the FP64 refinement done by FFT on a 128 x 128 grid
    g = synth.geom_ga64()
    prob = make_problem(g, seed=2)
    lams = synth.lambda_grid(16)
    rng = np.random.default_rng(5)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 2)])
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0] * 3, _lam_t(lams, 3), [16] * 3,
                           tol=1e-6, want_all_x=True, variant=5)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


def test_eval_fp32_fft_ragged_subpix(mods, ctx32):
    g = Geometry(30, 26, 0.09, 14, 12, -0.8, 0.8, -0.7, 0.7, 7, 2, REG_GRADIENT)
    prob = make_problem(g, seed=6)
    lams = synth.lambda_grid(8, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS, [1.1, 0.55, 2.0, -0.05, 0.04, 0.08, 2.5]]
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0, 0], _lam_t(lams, 2), [8, 8],
                           tol=1e-6, want_all_x=True, variant=5)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


def test_eval_fp64_fft_forced(mods, ctx64):
    # FP64 mode through the FP64 FFT: chi^2 to 1e-9 of the Cholesky oracle
    g = synth.geom_small_fp64()
    prob = make_problem(g, seed=1, psf_sigma=1.0)
    lams = synth.lambda_grid(10)
    lenses = [synth.TRUE_LENS, [0.95, 0.75, 0.4, 0.02, -0.03, 0.03, 0.8]]
    out = ctx64.eval_batch([device_problem(prob, torch.float64)], _lens_t(lenses), [0, 0], _lam_t(lams, 2),
                           [10, 10], tol=1e-12, maxit=50000, variant=5)
    for c, lens in enumerate(lenses):
        r = eval_candidate(prob, lens, lams)
        np.testing.assert_allclose(out["chi2"][c].cpu().numpy(), r.chi2, rtol=1e-9)
        assert int(out["corner"][c].item()) == r.corner


def test_fft_and_direct_agree_in_an_uneven_batch(mods, ctx32):
    # one call with a direct-convolution problem (9x9, on the two-CTA kernel)
    # and an FFT problem (41x41, automatic): every candidate matches the
    # oracle, in the mixed call and alone
    g1 = synth.geom_ga64()
    g2 = Geometry(48, 40, 0.07, 24, 20, -0.8, 0.8, -0.7, 0.7, 41, 1, REG_LAPLACIAN)
    p1, p2 = make_problem(g1, seed=2), make_problem(g2, seed=3, psf_sigma=5.0)
    lams = synth.lambda_grid(6, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS, [1.1, 0.6, 2.0, -0.05, 0.04, 0.08, 2.5], synth.TRUE_LENS]
    out = ctx32.eval_batch([device_problem(p1), device_problem(p2)], _lens_t(lenses), [0, 1, 1], _lam_t(lams, 3),
                           [6, 6, 6], tol=1e-6)
    for c, (pi, prob) in enumerate(((0, p1), (1, p2), (1, p2))):
        one = ctx32.eval_batch([device_problem(prob)], _lens_t([lenses[c]]), [0], _lam_t(lams, 1), [6], tol=1e-6)
        r = eval_candidate(prob, lenses[c], lams)
        np.testing.assert_allclose(out["chi2"][c].cpu().numpy(), r.chi2, rtol=2e-5)
        np.testing.assert_allclose(one["chi2"][0].cpu().numpy(), r.chi2, rtol=2e-5)
