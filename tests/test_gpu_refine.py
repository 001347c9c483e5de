"""Positivity source refinement (Section 3.2) on the forward batch: the GA
keeps its best, stays inside the paper's windows (hence non-negative), and
the chi^2 the library reports for its result is the oracle's."""
import numpy as np
import pytest
import torch

import synth
from oracle.solve import build_operators, forward_chi2

from .helpers import device_problem, make_problem

pytestmark = pytest.mark.gpu


def test_refine_keeps_best_within_windows():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.refine import RefineConfig, run_refine, windows

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    g = synth.geom_small_fp64()
    prob = make_problem(g, seed=31)
    dp = device_problem(prob)
    lens = synth.TRUE_LENS
    lam = torch.as_tensor(synth.lambda_grid(16)[None, :], device="cuda")
    out = ctx.eval_batch([dp], torch.as_tensor(lens[None, :], device="cuda"), [0], lam, [16], tol=1e-6)
    s_star = out["s"][0, :g.sx * g.sy].double().cpu().numpy()
    assert (s_star < 0).any()  # the regularised solution has negative pixels to fix
    n_fit = int((build_operators(prob, lens).w > 0).sum())
    hist, best, bchi = run_refine(ctx, dp, lens, s_star, n_fit, RefineConfig(pop=256, generations=30, seed=1))
    b = [h.best_chi2 for h in hist]
    assert all(b[i + 1] <= b[i] for i in range(len(b) - 1)), b
    lo, hi = windows(s_star)
    assert np.all(best >= lo - 1e-6) and np.all(best <= hi + 1e-6) and np.all(best >= 0)
    seed = np.clip(np.abs(s_star), lo, hi)
    seed_chi = float(forward_chi2(prob, lens, seed[None, :])[1][0])
    assert bchi <= seed_chi * (1 + 1e-5)
    ref = float(forward_chi2(prob, lens, best.astype(np.float32).astype(np.float64)[None, :])[1][0])
    assert abs(bchi - ref) <= 1e-5 * ref
    assert hist[-1].best_chi2_r == pytest.approx(bchi / (n_fit - g.sx * g.sy))
    ctx.close()
