"""Autotuner of the CGLS launch configuration of a shape class.

Three choices are tuned, each by timing a short probe batch with CUDA events
and keeping the fastest of a few runs:

* the kernel variant (mirage_opts_t.variant): the library's automatic
  choice (0), the two-CTA-per-SM kernel with PSF taps in shared memory (1),
  as kernel parameters with FFMA (2) or packed FFMA2 (3), and the general
  kernel (4), timed on the probe
  candidates at two lambdas from the middle of their grids (items of
  typical length);
* the reduction each inner solve of the refinement aims for
  (mirage_opts_t.inner_eta; FP32 contexts): a smaller target means fewer
  FP64 residual passes but longer inner solves, timed on the probe
  candidates' whole lambda grids, since the trade-off moves with lambda;
* the work-buffer placement and occupancy of the problems that run on the
  general kernel (mirage_opts_t.place): all in shared memory, the
  convolution inputs in shared memory and the rest in an L2-resident slab
  (one or two CTAs per SM), or all in the slab (one or two CTAs per SM).

A choice replaces the default only when it is more than MARGIN faster on the
probe (the placement: on the whole batch, where one evaluation of it is
cheap).  All choices solve the same systems to the same tolerance (variants
1-3 and the placements bitwise alike).  A shape class is the set of (image, source
grid, PSF, sub-pixels, regulariser) of the problems, the precision and
whether a launch mixes PSFs; its choice is cached in a JSON file and later
calls read the cache.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from .binding import MIRAGE_FP32

VARIANTS = (0, 1, 2, 3, 4)  # 0: the library's automatic choice
ETAS = (0.01, 0.03, 0.1)     # the first is the library's default
PLACES = (1, 2, 3, 4, 5)
MARGIN = 0.03                # a choice must beat the default by this much to replace it
MARGIN_PLACE = 0.05          # (a placement only moves the problems on the general kernel)
FULL_BATCH_MS = 5000.0       # placements are re-timed on whole batches up to this cost


def cache_path() -> str:
    p = os.environ.get("MIRAGE_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "mirage_gb300", "tune.json")


def shape_key(ctx, probs) -> str:
    gs = sorted({(int(p.geom.nx), int(p.geom.ny), int(p.geom.sx), int(p.geom.sy), int(p.geom.kpsf),
                  int(getattr(p.geom, "subpix", 1)), int(p.geom.reg)) for p in probs})
    return json.dumps({"prec": int(ctx.precision), "shapes": gs, "multi": len(probs) > 1})


def _load():
    try:
        return json.load(open(cache_path()))
    except Exception:
        return {}


def _save(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _time(ctx, probs, lens, prob_idx, lam, nl, reps, **kw) -> float:
    """Fastest of ``reps`` timed calls (after one warm-up), in ms."""
    ctx.eval_batch(probs, lens, prob_idx, lam, nl, **kw)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.eval_batch(probs, lens, prob_idx, lam, nl, **kw)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _pick(times: dict, default, margin=MARGIN):
    """The fastest choice, unless it beats the default by less than the
    margin (timing noise must not move a configuration)."""
    best = min(times, key=times.get)
    return best if times[best] < (1.0 - margin) * times[default] else default


def tune_config(ctx, probs, lens, prob_idx, lambdas, n_lam, *, tol=1e-6, n_probe=None, reps=3,
                retune=False, full_batch_ms=None) -> dict:
    """The fastest launch configuration for this shape class, as keyword
    arguments of ``Context.eval_batch`` (variant, inner_eta, place).  The
    probe is the first n_probe candidates (default 64, or 256 for classes of
    several problems, whose items vary more: a probe of a few items per CTA
    slot times the launch's tail, not its steady state).  The placement is
    then re-timed on the whole batch when one evaluation of it takes at most
    ``full_batch_ms`` (default FULL_BATCH_MS; 0: never)."""
    if full_batch_ms is None:
        full_batch_ms = FULL_BATCH_MS
    key = shape_key(ctx, probs)
    db = _load()
    if key in db and not retune and "inner_eta" in db[key]:
        e = db[key]
        return {"variant": int(e["variant"]), "inner_eta": float(e["inner_eta"]), "place": int(e["place"])}
    if n_probe is None:
        n_probe = 256 if len(probs) > 1 else 64
    n = min(n_probe, int(lens.shape[0]))
    m = int(lambdas.shape[1])
    pl = lens[:n].contiguous()
    pidx = prob_idx[:n]
    fp32 = ctx.precision == MIRAGE_FP32
    base = dict(tol=tol, want_s=False, want_kappa=False)
    # 1: the kernel variant, at two lambdas from the middle of the grids
    cols = [m // 2, min(m - 1, m // 2 + 1)] if m >= 2 else [0]
    lam2 = lambdas[:n, cols].contiguous()
    nl2 = np.minimum(np.asarray(n_lam[:n]), lam2.shape[1]).astype(np.int32)
    t_var = {}
    for v in VARIANTS:
        if v in (1, 2, 3) and not fp32:
            continue
        t_var[v] = _time(ctx, probs, pl, pidx, lam2, nl2, reps, variant=v, **base)
    variant = _pick(t_var, 0)
    # 2 and 3: on up to 256 candidates' whole grids (several items per CTA
    # slot, so that the launch's steady state, not its tail, is timed)
    n = min(max(n, 256), int(lens.shape[0]))
    pl = lens[:n].contiguous()
    pidx = prob_idx[:n]
    lam = lambdas[:n].contiguous()
    nl = np.asarray(n_lam[:n]).astype(np.int32)
    t_eta = {}
    eta = ETAS[0]
    if fp32:
        for e in ETAS:
            t_eta[e] = _time(ctx, probs, pl, pidx, lam, nl, reps, variant=variant, inner_eta=e, **base)
        eta = _pick(t_eta, ETAS[0])
    # (the two-CTA kernel has one layout: the placement only moves the
    # problems that run on the general kernel)
    t_place = {}
    for p in (0,) + PLACES:
        t_place[p] = _time(ctx, probs, pl, pidx, lam, nl, reps, variant=variant, inner_eta=eta, place=p, **base)
    place = _pick(t_place, 0, MARGIN_PLACE)
    # the placements again on the whole batch when that is cheap: how the
    # kernel groups of a mixed batch share the SMs (one or two CTAs per SM,
    # which groups overlap) depends on the batch's size, which a probe of a
    # few hundred candidates does not reproduce
    t_full = {}
    n_all = int(lens.shape[0])
    if n_all > n and full_batch_ms > 0:
        nl_all = np.asarray(n_lam).astype(np.int32)
        full = lambda p: _time(ctx, probs, lens, prob_idx, lambdas, nl_all, 1, variant=variant, inner_eta=eta,
                               place=p, **base)
        t_full[0] = full(0)
        if t_full[0] <= full_batch_ms:
            for p in PLACES:
                t_full[p] = full(p)
            place = _pick(t_full, 0, MARGIN)
    db[key] = {"variant": int(variant), "inner_eta": float(eta), "place": int(place),
               "ms": {"variant": {str(k): round(t, 4) for k, t in t_var.items()},
                      "inner_eta": {str(k): round(t, 4) for k, t in t_eta.items()},
                      "place": {str(k): round(t, 4) for k, t in t_place.items()},
                      "place_full_batch": {str(k): round(t, 4) for k, t in t_full.items()}}}
    _save(db)
    return {"variant": int(variant), "inner_eta": float(eta), "place": int(place)}


def tune(ctx, probs, lens, prob_idx, lambdas, n_lam, **kw) -> int:
    """The tuned kernel variant alone (see tune_config)."""
    return tune_config(ctx, probs, lens, prob_idx, lambdas, n_lam, **kw)["variant"]
