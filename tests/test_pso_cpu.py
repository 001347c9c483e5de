"""Host logic of the particle swarm (Eq. PSO): the periodic pull, the walls,
the stability of the two position updates, and convergence on a bowl."""
import numpy as np

import synth
from paper_1101_5803_gb300.pso import PSOConfig, confine, pso_step, run_pso, toward

LO, HI = synth.LENS_LO, synth.LENS_HI
MID = 0.5 * (LO + HI)


def test_toward_takes_the_short_way_round_for_angles():
    x = MID.copy()
    t = MID.copy()
    x[2], t[2] = 0.1, np.pi - 0.1       # phi: 0.2 apart across the wrap
    x[0], t[0] = 0.85, 1.15             # b: plain difference
    d = toward(x[None, :], t[None, :])[0]
    assert abs(d[2] - (-0.2)) < 1e-12
    assert abs(d[0] - 0.3) < 1e-12
    x[6], t[6] = 3.0, 0.05              # theta_g the other way
    assert abs(toward(x, t)[6] - (np.pi - 3.0 + 0.05)) < 1e-12


def test_confine_wraps_angles_and_reflects_the_rest():
    x = MID.copy()[None, :].repeat(3, axis=0)
    v = np.ones_like(x)
    x[0, 2] = np.pi + 0.3               # phi wraps to 0.3, velocity kept
    x[1, 0] = 1.25                      # b reflects at 1.2 to 1.15, velocity reversed
    x[2, 3] = -0.13                     # x0 reflects at -0.1 to -0.07
    xc, vc = confine(x, v)
    assert abs(xc[0, 2] - 0.3) < 1e-12 and vc[0, 2] == 1.0
    assert abs(xc[1, 0] - 1.15) < 1e-12 and vc[1, 0] == -1.0
    assert abs(xc[2, 3] - (-0.07)) < 1e-12 and vc[2, 3] == -1.0
    assert np.all(xc >= LO) and np.all(xc <= HI)
    # a step many box widths long still ends inside
    xf, _ = confine(MID + 50 * (HI - LO), np.ones(7))
    assert np.all(xf >= LO) and np.all(xf <= HI)


def _amplitude_after(explicit, steps=30):
    # one particle, both bests at the box centre, xi = 1/2: spring k = 1,
    # damping w = 1 - dt/t_damp = 0.75; start 1e-6 off centre in b
    cfg = PSOConfig(particles=1, explicit=explicit)
    x = MID.copy()[None, :]
    x[0, 0] += 1e-6
    v = np.zeros_like(x)
    half = np.full((1, 7), 0.5)
    amp = 0.0
    for _ in range(steps):
        x, v = pso_step(x, v, MID[None, :], MID, cfg, half, half)
        amp = abs(x[0, 0] - MID[0])
    return amp


def test_printed_update_is_unstable_and_new_velocity_update_is_not():
    # determinant of the step matrix: w + k = 1.75 (printed), w = 0.75 (default)
    assert _amplitude_after(explicit=True) > 1e-4      # grew by ~1.32 per step
    assert _amplitude_after(explicit=False) < 1e-7     # shrank by ~0.87 per step


def test_swarm_finds_the_minimum_of_a_bowl_across_the_wrap():
    target = MID.copy()
    target[2] = 0.02                    # phi next to the wrap
    target[0] = 1.13
    scale = HI - LO

    def evaluate(lens):
        d = toward(lens, target[None, :]) / scale
        f = (d ** 2).sum(axis=1)
        f[::17] = np.nan                # failed evaluations never become a best
        return f, 0

    hist, best, fbest = run_pso(evaluate, PSOConfig(particles=64, steps=80, seed=3))
    assert np.isfinite(fbest)
    assert fbest < 1e-6, fbest
    assert np.all(np.abs(toward(best, target)) < 2e-3 * scale)
    bests = [h.best_chi2 for h in hist]
    assert all(b1 <= b0 for b0, b1 in zip(bests, bests[1:]))
