"""Pins of the fixed-iteration CGLS oracle (Sections 2.4-2.6): each checks
it against something other than its own recursion.

* Krylov optimality: the k-th CGLS iterate from x_0 = 0 minimises ||b - A x||
  over the Krylov space span{A^T b, (A^T A) A^T b, ...} of dimension k; the
  minimiser is computed independently (QR basis + least squares).
* CGLS monotonicity: chi^2 never rises and ||x_k|| never falls.
* Convergence: with N_s unknowns and full column rank, the iterates reach the
  least-squares solution.
* Degrees of freedom: summed over unit vectors bhat = e_j on the fitted
  pixels, the twin's bhat^T (bhat - A xhat_k) is the trace of I - H_k; once
  the iteration has converged H is the projection onto range(A), whose trace
  is the column rank, so the sum is N_fit - N_s.
"""
import numpy as np
import pytest

import synth
from oracle.iterlc import cgls_iterations, weighted_system
from oracle.solve import build_operators
from synth import Geometry, REG_IDENTITY

from .helpers import make_problem


def _tiny(seed=3, nx=10, sx=4, interp=synth.INTERP_BILINEAR):
    g = Geometry(nx, nx, 0.16, sx, sx, -0.8, 0.8, -0.8, 0.8, 3, 1, REG_IDENTITY, interp=interp)
    return make_problem(g, seed=seed, psf_sigma=0.8)


def _krylov_minimiser(A, b, k):
    g = A.T @ b
    cols = [g]
    for _ in range(k - 1):
        cols.append(A.T @ (A @ cols[-1]))
    V, _ = np.linalg.qr(np.stack(cols, axis=1))
    y, *_ = np.linalg.lstsq(A @ V, b, rcond=None)
    return V @ y


@pytest.mark.parametrize("interp", [synth.INTERP_BILINEAR, synth.INTERP_NEAREST, synth.INTERP_BICUBIC])
def test_iterates_minimise_over_krylov_spaces(interp):
    prob = _tiny(interp=interp)
    ops = build_operators(prob, synth.TRUE_LENS)
    A, b = weighted_system(prob, ops)
    res = cgls_iterations(prob, synth.TRUE_LENS, 5, ops=ops)
    for k in range(1, 6):
        xk = _krylov_minimiser(A, b, k)
        assert np.linalg.norm(res.xs[k] - xk) <= 1e-8 * np.linalg.norm(xk), k


def test_chi2_falls_and_norm_rises():
    g = synth.geom_small_fp64()
    prob = make_problem(g, seed=4)
    res = cgls_iterations(prob, synth.TRUE_LENS, 30)
    assert np.all(np.diff(res.chi2) <= 1e-9 * res.chi2[0])
    assert np.all(np.diff(res.reg) >= -1e-9 * res.reg[-1])
    assert 1 <= res.corner <= 30


@pytest.mark.parametrize("interp", [synth.INTERP_BILINEAR, synth.INTERP_NEAREST, synth.INTERP_BICUBIC])
def test_iterates_reach_least_squares_solution(interp):
    prob = _tiny(seed=5, interp=interp)
    ops = build_operators(prob, synth.TRUE_LENS)
    A, b = weighted_system(prob, ops)
    assert np.linalg.matrix_rank(A) == A.shape[1]
    res = cgls_iterations(prob, synth.TRUE_LENS, 40, ops=ops)
    xls, *_ = np.linalg.lstsq(A, b, rcond=None)
    assert np.linalg.norm(res.xs[-1] - xls) <= 1e-7 * np.linalg.norm(xls)
    assert abs(res.chi2[-1] - float(np.sum((b - A @ xls) ** 2))) <= 1e-9 * res.chi2[0]


def test_twin_dof_sums_to_residual_rank():
    prob = _tiny(seed=6)
    ops = build_operators(prob, synth.TRUE_LENS)
    A, _ = weighted_system(prob, ops)
    ns = A.shape[1]
    assert np.linalg.matrix_rank(A) == ns
    fit = np.flatnonzero(ops.w > 0)
    n_iter = 40
    total = np.zeros(n_iter + 1)
    for j in fit:
        e = np.zeros(prob.d.size)
        e[j] = 1.0
        total += cgls_iterations(prob, synth.TRUE_LENS, n_iter, bhat=e.reshape(prob.d.shape), ops=ops).dof
    assert total[0] == pytest.approx(len(fit))
    assert abs(total[-1] - (len(fit) - ns)) <= 1e-6 * len(fit)


def test_gaussian_dof_estimate_is_unbiased():
    # the mean over standard-normal bhat matches the exact trace (unit vectors)
    prob = _tiny(seed=7)
    ops = build_operators(prob, synth.TRUE_LENS)
    fit = np.flatnonzero(ops.w > 0)
    k = 3
    exact = 0.0
    for j in fit:
        e = np.zeros(prob.d.size)
        e[j] = 1.0
        exact += cgls_iterations(prob, synth.TRUE_LENS, k, bhat=e.reshape(prob.d.shape), ops=ops).dof[k]
    rng = np.random.default_rng(11)
    est = [cgls_iterations(prob, synth.TRUE_LENS, k, bhat=rng.standard_normal(prob.d.shape), ops=ops).dof[k]
           for _ in range(400)]
    se = np.std(est) / np.sqrt(len(est))
    assert abs(np.mean(est) - exact) <= 4 * se + 1e-9
