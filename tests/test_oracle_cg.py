"""Pins of the matrix-free CGLS oracle (used where the dense F does not fit):
it reaches the dense Cholesky oracle's solution (a different algorithm on
the same system), and the normal-equation residual it reports is the one
recomputed from the dense operators."""
import numpy as np
import pytest

import synth
from oracle.cg import chi2_reg, cgls_solve, sparse_operators
from oracle.solve import build_operators, chi2_of, reg_of, solve_lambda

from .helpers import make_problem


@pytest.mark.parametrize("lam", [1e-2, 1.0])
def test_matrix_free_cgls_matches_cholesky(lam):
    g = synth.geom_small_fp64()
    prob = make_problem(g, seed=13)
    sops = sparse_operators(prob, synth.TRUE_LENS)
    s, rel, it = cgls_solve(sops, lam, tol=1e-12)
    assert rel <= 1e-12 and it > 0
    dops = build_operators(prob, synth.TRUE_LENS)
    s_ref = solve_lambda(dops, lam)
    assert np.linalg.norm(s - s_ref) <= 1e-8 * np.linalg.norm(s_ref)
    A = dops.FtWF + lam * dops.HtH
    assert np.linalg.norm(dops.rhs - A @ s) <= 2e-12 * np.linalg.norm(dops.rhs)
    c, r = chi2_reg(sops, s)
    assert c == pytest.approx(chi2_of(dops, prob.d, s), rel=1e-12)
    assert r == pytest.approx(reg_of(dops, s), rel=1e-12)
