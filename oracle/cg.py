"""Oracle: the regularised solve by matrix-free FP64 CGLS, for images whose
dense F = B L does not fit (256 x 256 and up).

Test infrastructure only (see ``oracle/__init__.py``).

The same system as ``oracle.solve`` (Eqs. chi2, eqLS and TKReg; Section 2.4
with x0 = 0), with the operators applied, never formed as products: L is the
sparse lens matrix, B the sparse blur matrix (the zero-padded convolution
that ``oracle.operators.blur_matrix`` builds and the dense oracle uses), W
the diagonal weights and H the sparse regulariser.  CGLS runs on the stacked
least-squares problem

    min || [sqrt(W) B L; sqrt(lam) H] s - [sqrt(W) d; 0] ||

until the normal-equation residual ||F^T W d - (F^T W F + lam H^T H) s||,
recomputed from s every 25 iterations, is at most tol ||F^T W d||.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .operators import blur_matrix, lens_matrix, reg_matrix, weight_vector
from .solve import Problem


@dataclasses.dataclass
class SparseOps:
    L: object
    B: object
    sw: np.ndarray   # sqrt(W)
    H: object
    b: np.ndarray    # sqrt(W) d
    rhs: np.ndarray  # F^T W d


def sparse_operators(prob: Problem, lens) -> SparseOps:
    L, mapped = lens_matrix(prob.geom, lens)
    B = blur_matrix(prob.geom, prob.psf, dense=False)
    sw = np.sqrt(weight_vector(prob.mask, mapped, prob.sigma))
    H = reg_matrix(prob.geom, prob.geom.reg)
    b = sw * np.asarray(prob.d, dtype=np.float64).ravel()
    rhs = L.T @ (B.T @ (sw * b))
    return SparseOps(L, B, sw, H, b, rhs)


def apply_F(ops: SparseOps, s):
    """sqrt(W) B L s."""
    return ops.sw * (ops.B @ (ops.L @ s))


def apply_Ft(ops: SparseOps, r):
    """L^T B^T sqrt(W) r."""
    return ops.L.T @ (ops.B.T @ (ops.sw * r))


def normal_residual(ops: SparseOps, s, lam: float):
    """F^T W d - (F^T W F + lam H^T H) s."""
    return ops.rhs - apply_Ft(ops, apply_F(ops, s)) - lam * (ops.H.T @ (ops.H @ s))


def cgls_solve(ops: SparseOps, lam: float, tol: float = 1e-12, maxit: int = 50000):
    """Returns (s, relative normal residual, iterations)."""
    ns = ops.L.shape[1]
    sl = np.sqrt(lam)
    x = np.zeros(ns)
    r1 = ops.b.copy()                 # image part of the stacked residual
    r2 = np.zeros(ops.H.shape[0])     # regulariser part
    s = apply_Ft(ops, r1) + sl * (ops.H.T @ r2)
    p = s.copy()
    gam = float(s @ s)
    rn = float(np.linalg.norm(ops.rhs))
    if rn == 0.0:
        return x, 0.0, 0
    rel = 1.0
    for it in range(1, maxit + 1):
        q1 = apply_F(ops, p)
        q2 = sl * (ops.H @ p)
        alpha = gam / float(q1 @ q1 + q2 @ q2)
        x += alpha * p
        r1 -= alpha * q1
        r2 -= alpha * q2
        s = apply_Ft(ops, r1) + sl * (ops.H.T @ r2)
        gnew = float(s @ s)
        p = s + (gnew / gam) * p
        gam = gnew
        if it % 25 == 0 or np.sqrt(gam) <= tol * rn:
            rel = float(np.linalg.norm(normal_residual(ops, x, lam))) / rn
            if rel <= tol:
                return x, rel, it
    return x, rel, maxit


def chi2_reg(ops: SparseOps, s):
    """(chi^2 of s, ||H s||^2)."""
    res = apply_F(ops, s) - ops.b
    hs = ops.H @ s
    return float(res @ res), float(hs @ hs)
