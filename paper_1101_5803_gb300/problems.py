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


def widepsf_workload(ctx: Context, n_cand: int = 16, n_lam: int = 8, k_psf: int = 65, seed: int = 0) -> Workload:
    """The 64x64 system with a wide PSF (the 65 x 65 class of the paper's
    large test): 64x64 image at 0.05"/px, 32x32 source over +-0.8", a
    k_psf x k_psf Gaussian PSF of sigma k_psf / 6 px, Laplacian H, n_lam
    lambdas log-spaced over 1e-3..1e1."""
    import dataclasses as _dc

    rng = np.random.default_rng(seed)
    g = _dc.replace(synth.geom_ga64(), kpsf=k_psf)
    psf = synth.gaussian_psf(k_psf, k_psf / 6.0)
    comps = synth.drawn_source(rng)
    prob = observe_on_device(ctx, g, psf, comps, synth.TRUE_LENS, rng)
    lens = torch.as_tensor(synth.lens_population(rng, n_cand), device="cuda")
    lams = torch.as_tensor(np.tile(synth.lambda_grid(n_lam, 1e-3, 1e1), (n_cand, 1)), device="cuda")
    return Workload(g, prob, lens, lams, np.full(n_cand, n_lam, np.int32), np.zeros(n_cand, np.int32))


def e2e128_workload(ctx: Context, n_cand: int = 512, n_lam: int = 16, seed: int = 0) -> Workload:
    """End-to-end GA system: 128x128 image at 0.03"/px, 48x48 source over
    +-0.8", 11x11 Gaussian PSF (sigma 1.5 px), Laplacian H, n_lam lambdas
    log-spaced over 1e-4..1e2."""
    rng = np.random.default_rng(seed)
    g = synth.geom_e2e128()
    psf = synth.gaussian_psf(g.kpsf, synth.PSF_SIGMA["e2e128"])
    prob = observe_on_device(ctx, g, psf, synth.drawn_source(rng), synth.TRUE_LENS, rng)
    lens = torch.as_tensor(synth.lens_population(rng, n_cand), device="cuda")
    lams = torch.as_tensor(np.tile(synth.lambda_grid(n_lam), (n_cand, 1)), device="cuda")
    return Workload(g, prob, lens, lams, np.full(n_cand, n_lam, np.int32), np.zeros(n_cand, np.int32))


@dataclasses.dataclass
class MultiWorkload:
    problems: list          # one Problem per distinct observation
    lens: torch.Tensor      # [n, 7] float64 (device)
    lambdas: torch.Tensor   # [n, max_lam] float64 (device)
    n_lam: np.ndarray       # [n] int32 (host)
    prob_idx: np.ndarray    # [n] int32 (host)


def uneven_workload(ctx: Context, n_cand: int = 1024, seed: int = 0) -> MultiWorkload:
    """Uneven persistent batch: every candidate has its own observation with an
    image of {48,64,96,128}^2 pixels over 6.4", an annular mask (inner
    0.3-0.6", outer 1.5-2.5"), a source grid of {16,24,32,48}^2 over +-0.8",
    a Gaussian PSF of width {7,11,15} px (sigma = width/6), and 8..32
    lambdas log-spaced over 1e-4..1e2."""
    rng = np.random.default_rng(seed)
    items = synth.uneven_batch(rng, n_cand)
    probs = []
    max_lam = max(it.n_lam for it in items)
    lams = np.zeros((n_cand, max_lam))
    for c, it in enumerate(items):
        psf = synth.gaussian_psf(it.geom.kpsf, it.psf_sigma)
        mask = synth.annular_mask(it.geom, it.r_in, it.r_out)
        probs.append(observe_on_device(ctx, it.geom, psf, synth.drawn_source(rng), synth.TRUE_LENS, rng, mask=mask))
        lams[c, :it.n_lam] = synth.lambda_grid(it.n_lam)
        lams[c, it.n_lam:] = lams[c, it.n_lam - 1]
    lens = torch.as_tensor(synth.lens_population(rng, n_cand), device="cuda")
    return MultiWorkload(probs, lens, torch.as_tensor(lams, device="cuda"),
                         np.array([it.n_lam for it in items], np.int32), np.arange(n_cand, dtype=np.int32))


def large_workload(ctx: Context, n_cand: int = 64, n_lam: int = 32, seed: int = 0) -> Workload:
    """Large field: 256x256 image at 0.02"/px, 128x128 source over +-1.2",
    21x21 Gaussian PSF (sigma 3 px), Laplacian H, n_lam lambdas."""
    rng = np.random.default_rng(seed)
    g = synth.geom_large256()
    psf = synth.gaussian_psf(g.kpsf, synth.PSF_SIGMA["large256"])
    prob = observe_on_device(ctx, g, psf, synth.drawn_source(rng), synth.TRUE_LENS, rng)
    lens = torch.as_tensor(synth.lens_population(rng, n_cand), device="cuda")
    lams = torch.as_tensor(np.tile(synth.lambda_grid(n_lam), (n_cand, 1)), device="cuda")
    return Workload(g, prob, lens, lams, np.full(n_cand, n_lam, np.int32), np.zeros(n_cand, np.int32))
