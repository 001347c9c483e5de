"""Device-resident synthetic lens problems for the benchmark and the GA.

The observed image is made on the GPU with the library's own forward model
(``mirage_forward``): the analytic source (``synth``) is sampled on a fine
160 x 160 source grid, traced through the true lens with 4 x 4 sub-pixels
per image pixel, blurred, and given Gaussian noise at S/N = 20 (peak over
sigma), the recipe of the paper's Section 2.3 test data.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

import synth

from .binding import Context, MIRAGE_FP32, Problem

FINE = 160  # fine source grid of the data model


@dataclasses.dataclass
class Workload:
    geom: object
    problem: Problem
    lens: torch.Tensor      # [n, 7] float64 (device)
    lambdas: torch.Tensor   # [n, n_lam] float64 (device)
    n_lam: np.ndarray       # [n] int32 (host)
    prob_idx: np.ndarray    # [n] int32 (host)


def observe_on_device(ctx: Context, geom, psf: np.ndarray, comps, lens_true, rng, snr: float = 20.0,
                      mask: np.ndarray | None = None) -> Problem:
    """Lensed, blurred, noisy image of an analytic source, made on the GPU."""
    dt = ctx.real
    dev = "cuda"
    ext = max(abs(geom.sxmin), abs(geom.sxmax), abs(geom.symin), abs(geom.symax))
    fine = dataclasses.replace(geom, sx=FINE, sy=FINE, sxmin=-ext, sxmax=ext, symin=-ext, symax=ext,
                               subpix=4)
    h = 2.0 * ext / FINE
    c = -ext + (np.arange(FINE) + 0.5) * h
    X, Y = np.meshgrid(c, c)
    sfine = synth.eval_source(comps, X, Y).ravel()
    npix = geom.nx * geom.ny
    zeros = torch.zeros(npix, dtype=dt, device=dev)
    ones = torch.ones(npix, dtype=dt, device=dev)
    allm = torch.ones(npix, dtype=torch.uint8, device=dev)
    psf_t = torch.as_tensor(psf.ravel(), dtype=dt, device=dev)
    pf = Problem(fine, zeros, ones, allm, psf_t)
    model, _, _ = ctx.forward(pf, torch.as_tensor(np.asarray(lens_true, dtype=np.float64), device=dev),
                              torch.as_tensor(sfine[None, :], dtype=dt, device=dev))
    clean = model[0]
    sigma_val = float(clean.abs().max().item()) / snr
    noise = torch.as_tensor(synth.standard_normal(rng, npix), dtype=dt, device=dev)
    d = clean + sigma_val * noise
    sigma = torch.full((npix,), sigma_val, dtype=dt, device=dev)
    m = allm if mask is None else torch.as_tensor(np.asarray(mask, dtype=np.uint8).ravel(), device=dev)
    return Problem(geom, d.contiguous(), sigma, m, psf_t)


def ga64_workload(ctx: Context, n_cand: int = 256, n_lam: int = 16, seed: int = 0) -> Workload:
    """Batched GA population: 64x64 image at 0.05"/px, 32x32 source over
    +-0.8", 9x9 Gaussian PSF (sigma 1.5 px), Laplacian H, n_cand lens vectors
    uniform in the search box, n_lam lambdas log-spaced over 1e-4..1e2."""
    rng = np.random.default_rng(seed)
    g = synth.geom_ga64()
    psf = synth.gaussian_psf(g.kpsf, synth.PSF_SIGMA["ga64"])
    comps = synth.drawn_source(rng)
    prob = observe_on_device(ctx, g, psf, comps, synth.TRUE_LENS, rng)
    lens = torch.as_tensor(synth.lens_population(rng, n_cand), device="cuda")
    lams = torch.as_tensor(np.tile(synth.lambda_grid(n_lam), (n_cand, 1)), device="cuda")
    return Workload(g, prob, lens, lams, np.full(n_cand, n_lam, np.int32), np.zeros(n_cand, np.int32))
