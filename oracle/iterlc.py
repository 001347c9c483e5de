"""Oracle: fixed-iteration CGLS, the L-curve over its iterations (Section
2.6) and the Monte Carlo degrees of freedom (Section 2.5), FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper's inner loop runs CGLS (Section 2.4) on the weighted
least-squares problem

    min_s || sqrt(W) (F s - d) ||,   F = B L,   W = diag(m / sigma^2),

from a blank source for a fixed number of iterations; the iteration count
acts as the regulariser (Section 2.4, implicit regularisation).  With
A = sqrt(W) F and b = sqrt(W) d, CGLS keeps the residual r = b - A x and the
normal-equation gradient s = A^T r:

    x_0 = 0, r_0 = b, s_0 = A^T b, p_0 = s_0, gamma_0 = ||s_0||^2
    q = A p_k,  alpha_k = gamma_k / ||q||^2
    x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k q
    s_{k+1} = A^T r_{k+1},  gamma_{k+1} = ||s_{k+1}||^2
    beta_k = gamma_{k+1} / gamma_k,  p_{k+1} = s_{k+1} + beta_k p_k

After every iteration the image chi^2 of x_k and the zeroth-order measure
sum x_k^2 are recorded (both evaluated from x_k itself, not from the
recursion); the corner of the L-curve through those points (oracle.lcurve)
selects the iteration whose chi^2 is the fitness.

Section 2.5: a twin run on a standard-normal vector bhat (restricted to the
pixels in the fit) reuses alpha_k and beta_k; bhat^T (bhat - A xhat_k)
estimates the residual degrees of freedom (the trace of I minus the
influence matrix of the frozen iteration).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .lcurve import lcurve_corner
from .solve import Operators, Problem, build_operators


@dataclasses.dataclass
class IterResult:
    chi2: np.ndarray      # [n_iter + 1]
    reg: np.ndarray       # [n_iter + 1] sum x_k^2
    dof: np.ndarray | None
    xs: np.ndarray        # [n_iter + 1, ns] iterates
    corner: int           # corner iteration, 1..n_iter
    kappa: np.ndarray     # [n_iter + 1], 0 at k = 0
    flat: bool


def weighted_system(prob: Problem, ops: Operators):
    """A = sqrt(W) F and b = sqrt(W) d of the weighted least-squares problem."""
    sw = np.sqrt(ops.w)
    return sw[:, None] * np.asarray(ops.F), sw * prob.d.ravel()


def cgls_iterations(prob: Problem, lens, n_iter: int, bhat=None, ops: Operators | None = None) -> IterResult:
    """n_iter CGLS iterations from x = 0 with per-iteration records, the
    iteration L-curve corner and, with ``bhat`` ([ny, nx]), the twin's dof."""
    ops = ops if ops is not None else build_operators(prob, lens)
    A, b = weighted_system(prob, ops)
    ns = A.shape[1]
    x = np.zeros(ns)
    r = b.copy()
    s = A.T @ r
    p = s.copy()
    gam = float(s @ s)
    chi2 = [float(b @ b)]
    reg = [0.0]
    xs = [x.copy()]
    twin = bhat is not None
    if twin:
        bh = np.where(ops.w > 0, np.asarray(bhat, dtype=np.float64).ravel(), 0.0)
        xh = np.zeros(ns)
        rh = bh.copy()
        ph = A.T @ rh
        dof = [float(bh @ bh)]
    for _ in range(n_iter):
        if not gam > 0:
            break
        q = A @ p
        alpha = gam / float(q @ q)
        x = x + alpha * p
        r = r - alpha * q
        s = A.T @ r
        gnew = float(s @ s)
        beta = gnew / gam
        gam = gnew
        p = s + beta * p
        res = b - A @ x
        chi2.append(float(res @ res))
        reg.append(float(x @ x))
        xs.append(x.copy())
        if twin:
            qh = A @ ph
            xh = xh + alpha * ph
            rh = rh - alpha * qh
            ph = A.T @ rh + beta * ph
            dof.append(float(bh @ (bh - A @ xh)))
    while len(chi2) < n_iter + 1:  # exact fit before n_iter: repeat the last record
        chi2.append(chi2[-1])
        reg.append(reg[-1])
        xs.append(xs[-1].copy())
        if twin:
            dof.append(dof[-1])
    cn, kap, flat = lcurve_corner(np.array(chi2[1:]), np.array(reg[1:]))
    return IterResult(np.array(chi2), np.array(reg), np.array(dof) if twin else None, np.array(xs), int(cn) + 1,
                      np.concatenate([[0.0], kap]), bool(flat))
