"""Genetic algorithm around the batched evaluator, with a learned screen.

The outer loop of Section 3 (the paper uses the Ferret GA, Appendix A.1):
a real-valued population inside a bounded search box, offspring made by
blend ("X-type") crossover along the line between two tournament-selected
parents (the fraction drawn from a Gaussian of width 0.25 about the
midpoint, so children may overshoot) and Gaussian mutation (probability
0.05 per gene, width 0.25 of the gene's range), and binary tournaments
between offspring and the parent population.  The fitness of a lens is the
chi^2 of its L-curve corner solution (Section 2.6).

With a surrogate, each generation draws ``oversample`` times more
offspring than it can afford exact solves for, ranks them by the
surrogate's predicted corner chi^2, evaluates the best ``pop`` exactly
(every survivor is judged by the exact solve) except for a control set of
``control * pop`` offspring drawn at random from the rest, and trains the
network on the new exact results.  The screen ranks, so its quality is
judged by the rank correlation between predicted and exact corner chi^2 on
the control set (the screened offspring alone span too narrow a range):
below ``fallback_rho`` the screen is switched off for the next generation
(offspring drawn without ranking), and back on when it recovers.  Warm-starting the children's CG from their parents' solutions
is available but off by default: a parent's source is a poor start for a
different lens and measured more CG iterations, not fewer.

With ``lam_chain`` the surrogate's predicted corner lambda also orders the
exact solves: each child's lambda grid is solved as two chains from the
grid point nearest the prediction, every lambda after a chain's first
starting from its neighbour's solution (fewer CG iterations, but chains are
serial work units, which costs parallelism on small populations).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

import synth

from .binding import MLP, Context
from .problems import Workload


def encode(lens: np.ndarray) -> np.ndarray:
    """Continuous features of lens vectors: the SIE is pi-periodic in phi and
    the shear in theta_g, so the angles enter through doubled-angle terms."""
    b, q, phi, x0, y0, g, tg = np.asarray(lens, dtype=np.float64).T
    return np.stack([b, (1 - q) * np.cos(2 * phi), (1 - q) * np.sin(2 * phi), x0, y0,
                     g * np.cos(2 * tg), g * np.sin(2 * tg)], axis=1)


@dataclasses.dataclass
class GAConfig:
    pop: int = 512
    generations: int = 20
    oversample: int = 4
    p_mutate: float = 0.05
    mutate_scale: float = 0.25
    xover_strength: float = 0.25
    tol: float = 1e-6
    surrogate: bool = True
    warm_start: bool = False
    lam_chain: bool = False
    hidden: int = 256
    train_steps: int = 200
    batch: int = 256
    lr: float = 2e-3
    fallback_rho: float = 0.3
    control: float = 0.125
    overlap_training: bool = True
    reserved_slots: int = 8
    seed: int = 0


@dataclasses.dataclass
class GenStats:
    gen: int
    best_chi2: float
    exact_evals: int
    decisions: int
    cg_iters: int
    seconds: float
    surrogate_rmse: float | None
    surrogate_rho: float | None
    screened: bool


class Surrogate:
    """Online-trained network mapping encoded lens -> standardised
    (log chi2*, log10 lambda*)."""

    def __init__(self, hidden: int, seed: int, device: int = 0):
        self.net = MLP([7, hidden, hidden, hidden, 2], device=device, seed=seed)
        self.X: list[np.ndarray] = []
        self.Y: list[np.ndarray] = []
        self.mu = self.sd = self.ymu = self.ysd = None

    def add(self, lens: np.ndarray, chi2: np.ndarray, lam: np.ndarray):
        ok = np.isfinite(chi2) & (chi2 > 0)
        self.X.append(encode(lens[ok]))
        self.Y.append(np.stack([np.log(chi2[ok]), np.log10(lam[ok])], axis=1))

    def _norm(self):
        X, Y = np.concatenate(self.X), np.concatenate(self.Y)
        self.mu, self.sd = X.mean(0), X.std(0) + 1e-9
        self.ymu, self.ysd = Y.mean(0), Y.std(0) + 1e-9
        return X, Y

    def train(self, steps: int, batch: int, lr: float, rng) -> None:
        """``steps`` Adam steps on minibatches of the rows gathered so far,
        drawn and run on the device in one library call."""
        X, Y = self._norm()
        xs = torch.as_tensor(((X - self.mu) / self.sd).astype(np.float32), device="cuda")
        ys = torch.as_tensor(((Y - self.ymu) / self.ysd).astype(np.float32), device="cuda")
        n = xs.shape[0]
        self.net.train(xs, ys, steps, min(batch, n), lr, seed=int(rng.integers(0, 2 ** 62)))

    def predict(self, lens: np.ndarray) -> np.ndarray:
        """Standardised predictions [n, 2] (log chi2*, log10 lambda*)."""
        x = torch.as_tensor(((encode(lens) - self.mu) / self.sd).astype(np.float32), device="cuda")
        return self.net.forward(x).cpu().numpy().astype(np.float64)

    def rmse(self, lens, chi2, lam) -> float:
        ok = np.isfinite(chi2) & (chi2 > 0)
        y = np.stack([np.log(chi2[ok]), np.log10(lam[ok])], axis=1)
        p = self.predict(lens[ok])
        return float(np.sqrt(np.mean(((y - self.ymu) / self.ysd - p) ** 2)))


def rank_corr(a, b) -> float:
    """Spearman rank correlation of two samples (no tie correction)."""
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def _offspring(pop: np.ndarray, fit: np.ndarray, n: int, cfg: GAConfig, rng):
    """n children by tournament selection, blend crossover, Gaussian mutation;
    returns (children, index of each child's first parent)."""
    lo, hi = synth.LENS_LO, synth.LENS_HI
    m = pop.shape[0]

    def tourney(k):
        a, b = rng.integers(0, m, k), rng.integers(0, m, k)
        return np.where(fit[a] <= fit[b], a, b)

    p1, p2 = tourney(n), tourney(n)
    r = 0.5 + cfg.xover_strength * rng.standard_normal((n, 1))
    kids = pop[p1] + r * (pop[p2] - pop[p1])
    mut = rng.uniform(size=kids.shape) < cfg.p_mutate
    kids = kids + mut * rng.standard_normal(kids.shape) * cfg.mutate_scale * (hi - lo)
    return np.clip(kids, lo, hi), p1


def run_ga(ctx: Context, wl: Workload, cfg: GAConfig, log=None):
    """Run the GA on one problem; returns (history, best lens, best chi2).

    With the surrogate and ``overlap_training``, the network trains on a
    side stream while each generation's exact solves run (the solve
    launches leave ``reserved_slots`` CTA slots free for it), on the exact
    results gathered up to the previous generation: the screen of
    generation g uses a network trained on generations 0..g-2, and the
    surrogate is off the solves' critical path."""
    rng = np.random.default_rng(cfg.seed)
    n_lam = int(wl.lambdas.shape[1])
    lam_row = wl.lambdas[0].cpu().numpy()
    pop = synth.lens_population(rng, cfg.pop)
    lam_dev = wl.lambdas[:1].expand(cfg.pop, n_lam).contiguous()
    probs = [wl.problem]
    pidx = np.zeros(cfg.pop, np.int32)
    nl = np.full(cfg.pop, n_lam, np.int32)
    sur = Surrogate(cfg.hidden, cfg.seed) if cfg.surrogate else None
    overlap = sur is not None and cfg.overlap_training
    side = torch.cuda.Stream() if overlap else None
    trained = [None]  # event recorded after the last training launch

    def launch(lens, warm, lam_start=None):
        return ctx.eval_batch(probs, torch.as_tensor(lens, device="cuda"), pidx, lam_dev, nl, tol=cfg.tol,
                              warm_x=warm, lam_start=lam_start, want_all_x=cfg.warm_start)

    def collect(lens, out):
        chi2 = out["chi2"].cpu().numpy()
        corner = out["corner"].cpu().numpy()
        fit = chi2[np.arange(len(lens)), corner]
        fit = np.where(np.isfinite(fit), fit, np.inf)
        return fit, lam_row[corner], out

    def train(steps):
        if not overlap:
            sur.train(steps, cfg.batch, cfg.lr, rng)
            return
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            sur.train(steps, cfg.batch, cfg.lr, rng)
            ev = torch.cuda.Event()
            ev.record(side)
        trained[0] = ev

    def predict(lens):
        # the network's buffers are shared by training and inference
        if trained[0] is not None:
            torch.cuda.current_stream().wait_event(trained[0])
        return sur.predict(lens)

    if overlap:
        ctx.reserve_slots(cfg.reserved_slots)
    try:
        t0 = time.perf_counter()
        fit, lam_star, out = collect(pop, launch(pop, None))
        X_pop = out["all_x"] if cfg.warm_start else None
        hist = [GenStats(0, float(fit.min()), cfg.pop, cfg.pop, int(out["iters"].sum().item()),
                         time.perf_counter() - t0, None, None, False)]
        if sur is not None:
            sur.add(pop, fit, lam_star)
            train(cfg.train_steps * (1 if overlap else 3))
        # with overlapped training the first network is still training beside
        # generation 1's solves, so generation 1 is drawn unscreened
        screen = sur is not None and not overlap
        for gen in range(1, cfg.generations + 1):
            t0 = time.perf_counter()
            n_draw = cfg.pop * (cfg.oversample if screen else 1)
            kids, par = _offspring(pop, fit, n_draw, cfg, rng)
            n_ctrl = 0
            if screen:
                # the pop - n_ctrl best-ranked offspring, plus n_ctrl drawn at
                # random from the rest: the control set on which the screen's
                # rank correlation and RMSE are measured without the range
                # restriction of its own selection
                pred = predict(kids)[:, 0]
                order = np.argsort(pred)
                n_ctrl = int(round(cfg.control * cfg.pop))
                top = order[:cfg.pop - n_ctrl]
                ctrl = rng.choice(order[cfg.pop - n_ctrl:], n_ctrl, replace=False)
                keep = np.concatenate([top, ctrl])
                kids, par = kids[keep], par[keep]
            warm = X_pop[par].contiguous() if cfg.warm_start else None
            lam_start = None
            if cfg.lam_chain and sur is not None and (screen or not overlap):
                # grid index nearest the predicted log10 lambda* of each child
                l10 = predict(kids)[:, 1] * sur.ysd[1] + sur.ymu[1]
                lam_start = np.abs(np.log10(lam_row)[None, :] - l10[:, None]).argmin(axis=1).astype(np.int32)
            if overlap and gen > 1:
                # on generations 0..gen-1, queued before this generation's
                # solves so that it runs beside them (the side stream waits
                # only for the work queued so far: the screen's inference)
                train(cfg.train_steps)
            kfit, klam, kout = collect(kids, launch(kids, warm, lam_start))
            rm = rho = None
            was_screened = screen
            if sur is not None:
                ok = np.isfinite(kfit) & (kfit > 0)
                if n_ctrl > 2:
                    ok[:cfg.pop - n_ctrl] = False  # judge the screen on its control set
                p = predict(kids)
                y = np.stack([np.log(kfit[ok]), np.log10(klam[ok])], axis=1)
                rm = float(np.sqrt(np.mean(((y - sur.ymu) / sur.ysd - p[ok]) ** 2)))
                rho = rank_corr(p[ok, 0], kfit[ok]) if ok.sum() > 2 else 0.0
                screen = rho >= cfg.fallback_rho
                sur.add(kids, kfit, klam)
                if not overlap:
                    train(cfg.train_steps)
            # binary tournaments between offspring and parents (mu + lambda)
            allp = np.concatenate([pop, kids])
            allf = np.concatenate([fit, kfit])
            allx = torch.cat([X_pop, kout["all_x"]]) if cfg.warm_start else None
            a = rng.permutation(cfg.pop)
            b = cfg.pop + rng.permutation(cfg.pop)
            win = np.where(allf[a] <= allf[b], a, b)
            # keep the best individual found so far
            best = int(np.argmin(allf))
            if best not in win:
                win[np.argmax(allf[win])] = best
            pop, fit = allp[win], allf[win]
            X_pop = allx[torch.as_tensor(win, device="cuda")].contiguous() if cfg.warm_start else None
            st = GenStats(gen, float(fit.min()), cfg.pop, n_draw, int(kout["iters"].sum().item()),
                          time.perf_counter() - t0, rm, rho, bool(was_screened))
            hist.append(st)
            if log:
                log(st)
    finally:
        if overlap:
            torch.cuda.synchronize()
            ctx.reserve_slots(0)
    b = int(np.argmin(fit))
    return hist, pop[b], float(fit[b])


def main(argv=None):
    """End-to-end GA on the 128x128 system (the surrogate-screened search):
    one JSON line per generation with the best corner chi^2, exact solves,
    offspring decisions, seconds, surrogate RMSE and rank correlation on the
    generation's exact results, and whether the screen was on (off = the
    fallback)."""
    import argparse
    import json

    from .binding import MIRAGE_FP32
    from .problems import e2e128_workload

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--pop", type=int, default=512)
    ap.add_argument("--generations", type=int, default=200)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--lam-chain", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    ctx = Context(0, MIRAGE_FP32)
    wl = e2e128_workload(ctx, n_cand=a.pop, seed=a.seed)
    cfg = GAConfig(pop=a.pop, generations=a.generations, surrogate=not a.no_surrogate, lam_chain=a.lam_chain,
                   seed=a.seed)

    def log(st):
        print(json.dumps({"gen": st.gen, "best_chi2": st.best_chi2, "exact_evals": st.exact_evals,
                          "decisions": st.decisions, "cg_iters": st.cg_iters, "seconds": round(st.seconds, 4),
                          "surrogate_rmse": st.surrogate_rmse, "surrogate_rho": st.surrogate_rho,
                          "screened": st.screened}), flush=True)

    hist, best, bchi = run_ga(ctx, wl, cfg, log=log)
    gens = hist[1:]
    print(json.dumps({"summary": True, "best_chi2": bchi, "best_lens": [float(v) for v in best],
                      "exact_evals_per_s": sum(h.exact_evals for h in gens) / sum(h.seconds for h in gens),
                      "fallback_rate": 1.0 - sum(h.screened for h in gens) / max(1, len(gens)),
                      "surrogate_rmse_last": gens[-1].surrogate_rmse if gens else None}), flush=True)


if __name__ == "__main__":
    main()
