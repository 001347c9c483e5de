"""The particle swarm on the batched evaluator (64x64 GA system): the global
best never gets worse, every step is one batched call, and the best
fitness is the corner chi^2 that a fresh evaluation of that lens gives."""
import numpy as np
import pytest

import synth

from .test_gpu_parity import ctx32, mods  # noqa: F401 (fixtures)

pytestmark = pytest.mark.gpu


def test_pso_on_the_batched_evaluator(mods, ctx32):
    from paper_1101_5803_gb300.problems import ga64_workload
    from paper_1101_5803_gb300.pso import PSOConfig, batch_evaluator, run_pso
    wl = ga64_workload(ctx32, n_cand=1, n_lam=16, seed=4)
    evaluate = batch_evaluator(ctx32, wl)
    calls = []

    def counted(lens):
        calls.append(lens.shape[0])
        return evaluate(lens)

    hist, best, fbest = run_pso(counted, PSOConfig(particles=128, steps=6, seed=1))
    assert calls == [128] * 7
    bests = [h.best_chi2 for h in hist]
    assert np.all(np.isfinite(bests))
    assert all(b1 <= b0 for b0, b1 in zip(bests, bests[1:]))
    assert bests[-1] < bests[0]
    assert np.all(best >= synth.LENS_LO) and np.all(best <= synth.LENS_HI)
    f_again, _ = evaluate(np.repeat(best[None, :], 2, axis=0))
    np.testing.assert_allclose(f_again, fbest, rtol=1e-5)
