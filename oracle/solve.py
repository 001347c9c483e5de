"""Oracle: the regularised semilinear solve by dense Cholesky (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

For one lens and one lambda (Eqs. chi2, eqLS and TKReg, Section 2.1, with
the default solution x0 = 0 of Eq. linsys, Section 2.4):

    F   = B L                              (f = B L, Section 2.1)
    A   = F^T W F + lambda H^T H           (M' = M + lambda H^T H)
    rhs = F^T W d                          (d' = F^T d / sigma^2)
    s   = A^{-1} rhs                       (dense Cholesky)
    chi2 = sum_j m_j (F s - d)_j^2 / sigma_j^2     (Eq. chi2)
    R    = ||H s||^2                        (regularisation measure)

The method reaches this solution exactly (up to the solver's tolerance), so
the oracle is the plain definition.  The L-curve corner over the lambda grid
is picked by ``oracle.lcurve``.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import scipy.linalg as sla

from .lcurve import lcurve_corner
from .operators import blur_matrix, lens_matrix, reg_matrix, weight_vector


@dataclasses.dataclass
class Problem:
    """One lens-inversion problem: geometry, data, noise map, mask and PSF."""

    geom: object
    d: np.ndarray       # [ny, nx]
    sigma: np.ndarray   # [ny, nx]
    mask: np.ndarray    # [ny, nx] uint8
    psf: np.ndarray     # [K, K]


@dataclasses.dataclass
class Operators:
    """Explicit operators of one (problem, lens) pair."""

    L: object
    mapped: np.ndarray
    B: object
    w: np.ndarray
    H: object
    F: np.ndarray
    FtWF: np.ndarray
    rhs: np.ndarray
    HtH: np.ndarray


def build_operators(prob: Problem, lens, timings: dict | None = None) -> Operators:
    """Assemble L, B, W, H, F = B L, F^T W F and F^T W d for one lens."""
    t0 = time.perf_counter()
    L, mapped = lens_matrix(prob.geom, lens)
    B = blur_matrix(prob.geom, prob.psf)
    w = weight_vector(prob.mask, mapped, prob.sigma)
    H = reg_matrix(prob.geom, prob.geom.reg)
    # F = B L, dense [npix, ns]
    F = np.asarray((L.T @ B.T).T) if isinstance(B, np.ndarray) else (B @ L).toarray()
    t1 = time.perf_counter()
    WF = F * w[:, None]
    FtWF = F.T @ WF
    rhs = WF.T @ np.asarray(prob.d, dtype=np.float64).ravel()
    HtH = (H.T @ H).toarray()
    t2 = time.perf_counter()
    if timings is not None:
        timings["build_F"] = timings.get("build_F", 0.0) + t1 - t0
        timings["FtWF"] = timings.get("FtWF", 0.0) + t2 - t1
    return Operators(L, mapped, B, w, H, F, FtWF, rhs, HtH)


def solve_lambda(ops: Operators, lam: float):
    """Cholesky solve of (F^T W F + lam H^T H) s = F^T W d."""
    A = ops.FtWF + lam * ops.HtH
    c = sla.cho_factor(A, lower=True, check_finite=False)
    return sla.cho_solve(c, ops.rhs, check_finite=False)


def _ld_matvec(M, x):
    """M x with products and sums in extended precision (np.longdouble)."""
    if isinstance(M, np.ndarray):
        return M.astype(np.longdouble) @ x
    return M.astype(np.longdouble) @ x


def normal_residual_ld(ops: Operators, prob: Problem, s, lam: float):
    """rhs - A s of Eq. TKReg's normal equations, from the factors L, B, W,
    H and d (not from the rounded products F^T W F and F^T W d), in
    extended precision."""
    ld = np.longdouble
    w = ops.w.astype(ld)
    d = np.asarray(prob.d, dtype=np.float64).ravel().astype(ld)
    x = np.asarray(s, dtype=np.float64).astype(ld)
    bls = _ld_matvec(ops.B, _ld_matvec(ops.L, x))
    img = w * (d - bls)
    ftwr = _ld_matvec(ops.L.T, _ld_matvec(ops.B.T, img))
    return ftwr - ld(lam) * _ld_matvec(ops.H.T, _ld_matvec(ops.H, x))


def solve_lambda_refined(ops: Operators, prob: Problem, lam: float, steps: int = 3):
    """The solution of (F^T W F + lam H^T H) s = F^T W d to near FP64
    rounding of s itself: the Cholesky solution, then classical iterative
    refinement (Wilkinson) with the residual formed in extended precision
    from the factors.  A plain FP64 Cholesky solve carries a forward error
    of order kappa_2(A) eps, which at kappa_2 ~ 1e5..1e7 is comparable to a
    1e-10 comparison; the refined solution does not."""
    A = ops.FtWF + lam * ops.HtH
    c = sla.cho_factor(A, lower=True, check_finite=False)
    s = sla.cho_solve(c, ops.rhs, check_finite=False)
    for _ in range(steps):
        r = normal_residual_ld(ops, prob, s, lam)
        ds = sla.cho_solve(c, np.asarray(r, dtype=np.float64), check_finite=False)
        s = np.asarray(s.astype(np.longdouble) + ds.astype(np.longdouble), dtype=np.float64)
    return s


def chi2_of(ops: Operators, d, s) -> float:
    """Eq. chi2 over pixels with m = 1 (folded into w)."""
    res = ops.F @ s - np.asarray(d, dtype=np.float64).ravel()
    return float(np.sum(ops.w * res * res))


def reg_of(ops: Operators, s) -> float:
    """Regularisation measure ||H s||^2."""
    hs = ops.H @ s
    return float(hs @ hs)


@dataclasses.dataclass
class EvalResult:
    chi2: np.ndarray     # [n_lam]
    reg: np.ndarray      # [n_lam]
    s: np.ndarray        # [n_lam, ns]
    corner: int
    kappa: np.ndarray    # [n_lam]
    mapped: np.ndarray   # [npix] bool
    timings: dict


def eval_candidate(prob: Problem, lens, lambdas) -> EvalResult:
    """Solve every lambda of the grid, then pick the L-curve corner."""
    timings: dict = {}
    ops = build_operators(prob, lens, timings)
    t0 = time.perf_counter()
    n = len(lambdas)
    S = np.zeros((n, prob.geom.ns))
    chi2 = np.zeros(n)
    reg = np.zeros(n)
    for k, lam in enumerate(lambdas):
        S[k] = solve_lambda(ops, float(lam))
        chi2[k] = chi2_of(ops, prob.d, S[k])
        reg[k] = reg_of(ops, S[k])
    t1 = time.perf_counter()
    corner, kappa, _ = lcurve_corner(chi2, reg)
    t2 = time.perf_counter()
    timings["cholesky"] = t1 - t0
    timings["lcurve"] = t2 - t1
    return EvalResult(chi2, reg, S, corner, kappa, ops.mapped, timings)


def forward_chi2(prob: Problem, lens, S):
    """Forward model B L s and its chi2 for a batch of sources S [n, ns]."""
    ops = build_operators(prob, lens)
    S = np.atleast_2d(np.asarray(S, dtype=np.float64))
    model = S @ ops.F.T
    res = model - np.asarray(prob.d, dtype=np.float64).ravel()[None, :]
    return model, np.sum(ops.w[None, :] * res * res, axis=1)
