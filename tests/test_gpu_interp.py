"""GPU parity of the other source interpolations (geometry field ``interp``)
against the FP64 oracle.

Section 2.1 lists nearest-neighbour and bicubic interpolation beside
bilinear.  Nearest neighbour puts each ray's whole weight on the closest
centre; bicubic spreads it over the 4 x 4 centres around the ray's cell with
Keys' cubic-convolution kernel.  Both sides trace the rays in FP64 and take
the cell and offsets from the same FP64 numbers, so the operator is the same
matrix on both (bicubic weights are evaluated in the context's precision).
The gates are those of the bilinear tests: the forward model to float
rounding, every lambda's solve by its normal-equation residual, chi^2
against the oracle's, and the corner.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
from oracle.iterlc import cgls_iterations
from oracle.lcurve import lcurve_corner
from oracle.operators import lens_matrix
from oracle.solve import eval_candidate, forward_chi2
from synth import Geometry, REG_GRADIENT, REG_LAPLACIAN

from .helpers import device_problem, make_problem
from .test_gpu_parity import _fp32_checks, _lam_t, _lens_t, ctx32, ctx64, mods  # noqa: F401 (fixtures)

pytestmark = pytest.mark.gpu


INTERPS = [synth.INTERP_NEAREST, synth.INTERP_BICUBIC]


def _with(g, interp):
    return dataclasses.replace(g, interp=interp)


def _operator_is_the_asked_one(prob, lens):
    """The oracle's L for this geometry has the asked structure (a sanity
    check that the test exercises the option, not bilinear): one centre per
    ray for nearest neighbour, more than the bilinear four for bicubic."""
    L, _ = lens_matrix(prob.geom, lens)
    L = L.tocsr()
    L.eliminate_zeros()
    nnz_per_row = np.diff(L.indptr)
    if prob.geom.interp == synth.INTERP_NEAREST:
        return nnz_per_row.max() <= prob.geom.subpix ** 2
    return nnz_per_row.max() > 4 * prob.geom.subpix ** 2 or np.median(nnz_per_row[nnz_per_row > 0]) > 4


@pytest.mark.parametrize("interp", INTERPS)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("geom", [
    Geometry(30, 27, 0.09, 11, 13, -0.9, 0.7, -0.8, 0.9, 7, 2, REG_GRADIENT),   # ragged, sub-pixels
    Geometry(64, 64, 0.05, 32, 32, -0.8, 0.8, -0.8, 0.8, 9, 1, REG_LAPLACIAN),
    Geometry(96, 90, 0.034, 48, 40, -0.8, 0.8, -0.7, 0.7, 21, 1, REG_LAPLACIAN),  # banded kernel
])
def test_forward_matches_oracle(mods, ctx32, ctx64, precision, geom, interp):
    geom = _with(geom, interp)
    ctx = ctx32 if precision == "fp32" else ctx64
    dt = torch.float32 if precision == "fp32" else torch.float64
    prob = make_problem(geom, seed=13)
    lens = [1.05, 0.65, 0.3, 0.03, -0.02, 0.04, 0.7]
    assert _operator_is_the_asked_one(prob, lens)
    S = np.random.default_rng(14).uniform(0, 1, (6, geom.ns))
    m_o, c_o = forward_chi2(prob, lens, S)
    m_g, c_g, st = ctx.forward(device_problem(prob, dt), _lens_t(lens)[0],
                               torch.as_tensor(S, dtype=dt, device="cuda"))
    tol = 2e-6 if precision == "fp32" else 1e-12
    assert int(st.item()) == 0
    m_g = m_g.double().cpu().numpy()
    assert np.abs(m_g - m_o).max() <= tol * np.abs(m_o).max()
    np.testing.assert_allclose(c_g.cpu().numpy(), c_o, rtol=50 * tol)


@pytest.mark.parametrize("interp", INTERPS)
def test_forward_differs_from_bilinear(mods, ctx64, interp):
    # the option reaches the kernels: the two models of one source differ
    g = Geometry(64, 64, 0.05, 32, 32, -0.8, 0.8, -0.8, 0.8, 9, 1, REG_LAPLACIAN)
    prob_b = make_problem(g, seed=13)
    prob_n = dataclasses.replace(prob_b, geom=_with(g, interp))
    lens = _lens_t([1.05, 0.65, 0.3, 0.03, -0.02, 0.04, 0.7])[0]
    S = torch.as_tensor(np.random.default_rng(1).uniform(0, 1, (1, g.ns)), device="cuda")
    m_b, _, _ = ctx64.forward(device_problem(prob_b, torch.float64), lens, S)
    m_n, _, _ = ctx64.forward(device_problem(prob_n, torch.float64), lens, S)
    assert (m_b - m_n).abs().max().item() > 1e-4 * m_b.abs().max().item()


@pytest.mark.parametrize("interp,variant", [(synth.INTERP_NEAREST, 0), (synth.INTERP_NEAREST, 4),
                                            (synth.INTERP_BICUBIC, 0)])
def test_eval_fp32_64px(mods, ctx32, interp, variant):
    # the 64x64 system of the GA batch: fast kernel (variant 0; bicubic runs
    # on the general kernel whatever the variant) and general kernel
    # (variant 4), 16 lambdas, tol 1e-6
    g = _with(synth.geom_ga64(), interp)
    prob = make_problem(g, seed=2)
    lams = synth.lambda_grid(16)
    rng = np.random.default_rng(5)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 2)])
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0] * 3, _lam_t(lams, 3), [16] * 3,
                           tol=1e-6, want_all_x=True, variant=variant)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


@pytest.mark.parametrize("interp", INTERPS)
def test_eval_fp32_ragged_subpix(mods, ctx32, interp):
    g = _with(Geometry(30, 26, 0.09, 14, 12, -0.8, 0.8, -0.7, 0.7, 7, 2, REG_GRADIENT), interp)
    prob = make_problem(g, seed=6)
    lams = synth.lambda_grid(8, 1e-3, 1e1)
    lenses = [synth.TRUE_LENS, [1.1, 0.55, 2.0, -0.05, 0.04, 0.08, 2.5]]
    out = ctx32.eval_batch([device_problem(prob)], _lens_t(lenses), [0, 0], _lam_t(lams, 2), [8, 8],
                           tol=1e-6, want_all_x=True)
    _fp32_checks(out, prob, lenses, lams, 1e-6)


@pytest.mark.parametrize("interp", INTERPS)
def test_eval_fp64_grid_and_corner(mods, ctx64, interp):
    g = _with(synth.geom_small_fp64(), interp)
    prob = make_problem(g, seed=1, psf_sigma=1.0)
    lams = synth.lambda_grid(10)
    lenses = [synth.TRUE_LENS, [0.95, 0.75, 0.4, 0.02, -0.03, 0.03, 0.8]]
    out = ctx64.eval_batch([device_problem(prob, torch.float64)], _lens_t(lenses), [0, 0], _lam_t(lams, 2),
                           [10, 10], tol=1e-12, maxit=50000)
    for c, lens in enumerate(lenses):
        r = eval_candidate(prob, lens, lams)
        np.testing.assert_allclose(out["chi2"][c].cpu().numpy(), r.chi2, rtol=1e-9)
        np.testing.assert_allclose(out["reg"][c].cpu().numpy(), r.reg, rtol=1e-6)
        assert int(out["corner"][c].item()) == r.corner


@pytest.mark.parametrize("interp", INTERPS)
def test_iter_lcurve_fp64(mods, ctx64, interp):
    # the fixed-iteration L-curve with the other interpolations.  Unique: the first
    # iterations, before CGLS loses orthogonality (after that two correct FP64
    # runs drift apart).  Checked as valid: the corner is the one the oracle's
    # corner rule picks from the library's own records.
    g = _with(synth.geom_small_fp64(), interp)
    prob = make_problem(g, seed=21)
    rng = np.random.default_rng(3)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 2)])
    n_iter = 30
    out = ctx64.eval_iter([device_problem(prob, torch.float64)], _lens_t(lenses), [0] * len(lenses), n_iter)
    for c, lens in enumerate(lenses):
        r = cgls_iterations(prob, lens, n_iter)
        chi = out["chi2"][c].cpu().numpy()
        assert np.all(np.abs(chi[:7] / r.chi2[:7] - 1) <= 1e-12), (c, chi[:7], r.chi2[:7])
        reg = out["reg"][c].cpu().numpy()
        cn = lcurve_corner(chi[1:], reg[1:])[0] + 1
        assert int(out["corner"][c]) == cn, (c, int(out["corner"][c]), cn, r.corner)
