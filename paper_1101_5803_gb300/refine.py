"""Positivity source refinement (Section 3.2) on the batched forward model.

With the lens held fixed, every source pixel becomes a bounded parameter of
a GA whose fitness is the image chi^2 of B L s; one ``mirage_forward`` call
evaluates a whole generation.  The bounds are the paper's windows around the
optimally regularised solution s*: [0.75 s*_i, 1.25 s*_i] where s*_i >= 0 and
[0, 1.15 |s*_i|] where s*_i < 0, so the refined source is non-negative; |s*|
(clipped into its window) is seeded into the first generation.  There is no
regulariser, so the degrees of freedom are N_fit - N_s and
chi^2_r = chi^2 / (N_fit - N_s).

The GA operators are those of ``ga.py`` (tournament selection, blend
crossover of width ``xover_strength`` about the midpoint, Gaussian mutation
of ``mutate_scale`` times the window width with probability ``p_mutate`` per
pixel, binary tournaments between children and parents) with the best
individual always kept.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from .binding import Context


def windows(s_star, tol: float = 0.25, neg_up: float = 0.15):
    """Per-pixel bounds (lo, hi) of the refinement around s* (Section 3.2)."""
    s = np.asarray(s_star, dtype=np.float64)
    pos = s >= 0
    lo = np.where(pos, (1.0 - tol) * s, 0.0)
    hi = np.where(pos, (1.0 + tol) * s, (1.0 + neg_up) * np.abs(s))
    return lo, hi


@dataclasses.dataclass
class RefineConfig:
    pop: int = 1024
    generations: int = 200
    p_mutate: float = 0.05
    mutate_scale: float = 0.25
    xover_strength: float = 0.25
    seed: int = 0


@dataclasses.dataclass
class RefineStats:
    gen: int
    best_chi2: float
    best_chi2_r: float
    seconds: float


def run_refine(ctx: Context, prob, lens, s_star, n_fit: int, cfg: RefineConfig, log=None):
    """Refine the source at a fixed lens; returns (history, best source, best chi^2)."""
    rng = np.random.default_rng(cfg.seed)
    lo, hi = windows(s_star)
    ns = lo.size
    width = hi - lo
    dof = max(1, int(n_fit) - ns)
    lens_t = torch.as_tensor(np.asarray(lens, dtype=np.float64), device="cuda")
    dt = ctx.real

    def fitness(pop):
        _, chi2, _ = ctx.forward(prob, lens_t, torch.as_tensor(pop, dtype=dt, device="cuda"), want_model=False)
        return chi2.cpu().numpy()

    pop = lo + rng.uniform(size=(cfg.pop, ns)) * width
    pop[0] = np.clip(np.abs(np.asarray(s_star, dtype=np.float64)), lo, hi)
    fit = fitness(pop)
    hist = [RefineStats(0, float(fit.min()), float(fit.min()) / dof, 0.0)]
    for gen in range(1, cfg.generations + 1):
        t0 = time.perf_counter()
        m = cfg.pop
        a, b = rng.integers(0, m, (2, m)), rng.integers(0, m, (2, m))
        p1 = np.where(fit[a[0]] <= fit[b[0]], a[0], b[0])
        p2 = np.where(fit[a[1]] <= fit[b[1]], a[1], b[1])
        r = 0.5 + cfg.xover_strength * rng.standard_normal((m, 1))
        kids = pop[p1] + r * (pop[p2] - pop[p1])
        mut = rng.uniform(size=kids.shape) < cfg.p_mutate
        kids = kids + mut * rng.standard_normal(kids.shape) * cfg.mutate_scale * width
        kids = np.clip(kids, lo, hi)
        kfit = fitness(kids)
        allp = np.concatenate([pop, kids])
        allf = np.concatenate([fit, kfit])
        ia = rng.permutation(m)
        ib = m + rng.permutation(m)
        win = np.where(allf[ia] <= allf[ib], ia, ib)
        best = int(np.argmin(allf))
        if best not in win:
            win[np.argmax(allf[win])] = best
        pop, fit = allp[win], allf[win]
        st = RefineStats(gen, float(fit.min()), float(fit.min()) / dof, time.perf_counter() - t0)
        hist.append(st)
        if log:
            log(st)
    b = int(np.argmin(fit))
    return hist, pop[b], float(fit[b])
