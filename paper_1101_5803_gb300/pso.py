"""Particle swarm around the batched evaluator (Section 3.1's PSO, Eq. PSO).

Each particle is a lens vector in the same search box as the GA.  Every
step the whole swarm is one batched evaluation: the fitness of a lens is
the chi^2 of its L-curve corner solution (Section 2.6).  The velocity
follows Eq. PSO: the old velocity damped by (1 - dt / t_damp), plus spring
pulls towards the particle's personal best and the swarm's global best,
each scaled by its constant (c_p, c_g) and a uniform random factor in
[0, 1) drawn per particle and per parameter.  The position advances by the
new velocity (the standard PSO update; the paper takes the velocity as
constant over a step).  The equation as printed advances it by the
velocity of the start of the step instead (``explicit=True``).  That form
is unstable for the usual constants: for one coordinate pulled towards a
fixed best with spring k and damping factor w = 1 - dt/t_damp, the step
matrix has determinant w + k, so with k ~ 1 the swarm oscillates with
growing amplitude.  The new-velocity form has determinant w.

The search box has two kinds of wall.  The SIE orientation phi and the
shear angle theta_g are pi-periodic (the model repeats), so they wrap
around, and a pull towards a best solution takes the shorter way round.
The other parameters reflect at the walls, and the velocity component
reverses with them.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

import synth

PERIODIC = np.array([False, False, True, False, False, False, True])  # phi, theta_g


@dataclasses.dataclass
class PSOConfig:
    particles: int = 512
    steps: int = 50
    dt: float = 1.0
    t_damp: float = 4.0
    c_p: float = 1.0
    c_g: float = 1.0
    v0: float = 0.1       # initial speeds: uniform in +-v0 of each parameter's range
    explicit: bool = False  # advance positions by the old velocity (Eq. PSO as printed)
    tol: float = 1e-6
    seed: int = 0


@dataclasses.dataclass
class StepStats:
    step: int
    best_chi2: float
    evals: int
    cg_iters: int
    seconds: float


def toward(x, target, lo=synth.LENS_LO, hi=synth.LENS_HI):
    """target - x, with the periodic parameters taking the shorter way round."""
    d = np.asarray(target, dtype=np.float64) - np.asarray(x, dtype=np.float64)
    span = hi - lo
    wrapped = d - span * np.round(d / span)
    return np.where(PERIODIC, wrapped, d)


def confine(x, v, lo=synth.LENS_LO, hi=synth.LENS_HI):
    """Wrap the periodic parameters into [lo, hi) and reflect the others at
    the walls (reversing the velocity component); returns (x, v)."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    span = hi - lo
    per = np.broadcast_to(PERIODIC, x.shape)
    x = np.where(per, lo + np.mod(x - lo, span), x)
    for _ in range(4):  # a step longer than the box folds more than once
        below, above = (x < lo) & ~per, (x > hi) & ~per
        if not (below.any() or above.any()):
            break
        x = np.where(below, 2 * lo - x, np.where(above, 2 * hi - x, x))
        v = np.where(below | above, -v, v)
    return np.clip(x, lo, hi), v


def pso_step(x, v, x_p, x_g, cfg: PSOConfig, xi_p, xi_g):
    """One step of Eq. PSO for the whole swarm: [n, 7] positions x and
    velocities v, personal bests x_p [n, 7], global best x_g [7], uniform
    factors xi_p, xi_g [n, 7].  Returns the confined (x, v) after the step."""
    pull = cfg.c_p * xi_p * toward(x, x_p) + cfg.c_g * xi_g * toward(x, x_g[None, :])
    v_new = v * (1.0 - cfg.dt / cfg.t_damp) + pull * cfg.dt
    x_new = x + (v if cfg.explicit else v_new) * cfg.dt
    return confine(x_new, v_new)


def run_pso(evaluate, cfg: PSOConfig, log=None):
    """Run the swarm with ``evaluate(lens [n, 7]) -> (fitness [n], cg_iters)``
    (lower is better; non-finite fitness never becomes a best).  Returns
    (history, best lens, best fitness)."""
    rng = np.random.default_rng(cfg.seed)
    lo, hi = synth.LENS_LO, synth.LENS_HI
    n = cfg.particles
    t0 = time.perf_counter()
    x = synth.lens_population(rng, n)
    v = rng.uniform(-cfg.v0, cfg.v0, size=(n, 7)) * (hi - lo)
    fit, iters = evaluate(x)
    fit = np.where(np.isfinite(fit), fit, np.inf)
    x_p, f_p = x.copy(), fit.copy()
    g = int(np.argmin(f_p))
    x_g, f_g = x_p[g].copy(), float(f_p[g])
    hist = [StepStats(0, f_g, n, iters, time.perf_counter() - t0)]
    if log:
        log(hist[-1])
    for step in range(1, cfg.steps + 1):
        t0 = time.perf_counter()
        xi_p = rng.uniform(size=(n, 7))
        xi_g = rng.uniform(size=(n, 7))
        x, v = pso_step(x, v, x_p, x_g, cfg, xi_p, xi_g)
        fit, iters = evaluate(x)
        fit = np.where(np.isfinite(fit), fit, np.inf)
        better = fit < f_p
        x_p[better], f_p[better] = x[better], fit[better]
        g = int(np.argmin(f_p))
        if f_p[g] < f_g:
            x_g, f_g = x_p[g].copy(), float(f_p[g])
        hist.append(StepStats(step, f_g, n, iters, time.perf_counter() - t0))
        if log:
            log(hist[-1])
    return hist, x_g, f_g


def batch_evaluator(ctx, wl, tol: float = 1e-6):
    """``evaluate`` for ``run_pso``: the corner chi^2 of each lens on one
    problem by one batched call of the exact evaluator."""
    import torch

    n_lam = int(wl.lambdas.shape[1])
    probs = [wl.problem]

    def evaluate(lens):
        m = lens.shape[0]
        lam = wl.lambdas[:1].expand(m, n_lam).contiguous()
        out = ctx.eval_batch(probs, torch.as_tensor(lens, device="cuda"), np.zeros(m, np.int32), lam,
                             np.full(m, n_lam, np.int32), tol=tol)
        chi2 = out["chi2"].cpu().numpy()
        corner = out["corner"].cpu().numpy()
        return chi2[np.arange(m), corner], int(out["iters"].sum().item())

    return evaluate


def main(argv=None):
    """Particle swarm on the 128x128 system: one JSON line per step with the
    global best corner chi^2, exact solves, CG iterations and seconds."""
    import argparse
    import json

    from .binding import MIRAGE_FP32, Context
    from .problems import e2e128_workload

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--particles", type=int, default=512)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    ctx = Context(0, MIRAGE_FP32)
    wl = e2e128_workload(ctx, n_cand=a.particles, seed=a.seed)
    cfg = PSOConfig(particles=a.particles, steps=a.steps, seed=a.seed)

    def log(st):
        print(json.dumps({"step": st.step, "best_chi2": st.best_chi2, "exact_evals": st.evals,
                          "cg_iters": st.cg_iters, "seconds": round(st.seconds, 4)}), flush=True)

    hist, best, bchi = run_pso(batch_evaluator(ctx, wl, cfg.tol), cfg, log=log)
    steps = hist[1:]
    print(json.dumps({"summary": True, "best_chi2": bchi, "best_lens": [float(t) for t in best],
                      "exact_evals_per_s": sum(h.evals for h in steps) / max(1e-9, sum(h.seconds for h in steps))}),
          flush=True)


if __name__ == "__main__":
    main()
