"""What the trained surrogate gains over the GA without it.

Offspring of a GA population are drawn four times over and ALL are solved
exactly; the surrogate (trained on a few generations of exact results)
then picks a quarter of them.  Its picks must have a clearly lower exact
corner chi^2 than an equal random quarter, and its ranking must correlate
with the exact one.  Without the surrogate the GA would spend its exact
solves on the random quarter.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_screen_picks_better_offspring():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.ga import GAConfig, Surrogate, _offspring, rank_corr
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    N = 128
    wl = ga64_workload(ctx, 4 * N, 16, seed=77)
    lam_row = wl.lambdas[0].cpu().numpy()

    def evaluate(lens):
        n = len(lens)
        out = ctx.eval_batch([wl.problem], torch.as_tensor(lens, device="cuda"), np.zeros(n, np.int32),
                             wl.lambdas[:n].contiguous(), np.full(n, 16, np.int32), tol=1e-6)
        chi2, corner = out["chi2"].cpu().numpy(), out["corner"].cpu().numpy()
        return chi2[np.arange(n), corner], lam_row[corner]

    rng = np.random.default_rng(11)
    cfg = GAConfig(pop=N, seed=11)
    sur = Surrogate(256, 3)
    pop = synth.lens_population(rng, N)
    fit, lam = evaluate(pop)
    sur.add(pop, fit, lam)
    sur.train(600, 256, 2e-3, rng)
    gains, rhos = [], []
    for gen in range(4):
        kids, _ = _offspring(pop, fit, 4 * N, cfg, rng)
        kfit, klam = evaluate(kids)
        pred = sur.predict(kids)[:, 0]
        top = np.argsort(pred)[:N]
        rnd = rng.permutation(4 * N)[:N]
        gains.append(np.median(kfit[rnd]) / np.median(kfit[top]))
        rhos.append(rank_corr(pred, kfit))
        sur.add(kids, kfit, klam)
        sur.train(200, 256, 2e-3, rng)
        allp, allf = np.concatenate([pop, kids]), np.concatenate([fit, kfit])
        keep = np.argsort(allf)[:N]
        pop, fit = allp[keep], allf[keep]
    ctx.close()
    # after the first generations of training the screen's picks are
    # clearly better than random picks of the same offspring
    assert np.mean(gains[1:]) > 1.1, gains
    assert np.mean(rhos[1:]) > 0.4, rhos


def test_ga_with_lambda_chains():
    # the GA with the surrogate's predicted corner ordering the exact solves
    # (lambda chains): every fitness finite, the best chi^2 never rises
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.ga import GAConfig, run_ga
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, 64, 16, seed=5)
    hist, best, bchi = run_ga(ctx, wl, GAConfig(pop=64, generations=2, lam_chain=True, train_steps=50, seed=3))
    assert np.isfinite(bchi) and len(best) == 7
    b = [h.best_chi2 for h in hist]
    assert all(b[i + 1] <= b[i] for i in range(len(b) - 1)), b
    assert all(h.cg_iters > 0 for h in hist)
