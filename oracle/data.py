"""Oracle: synthetic lensed observations (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

As in the paper's test problems (Section 2.3): the analytic source is
sampled through the lens at a finer sub-pixel grid than the model uses (here
4 x 4 sub-pixels per image pixel, surface brightness conserved per ray,
Eq. consSurfB), averaged per pixel, blurred by the PSF and given additive
Gaussian noise with S/N = peak / sigma (the paper's S/N definition).
"""
from __future__ import annotations

import numpy as np
from scipy.signal import convolve2d

from synth import eval_source

from .lens import ray_trace
from .operators import image_centres, subpixel_offsets
from .solve import Problem


def lensed_image(geom, lens, comps, nsub: int = 4) -> np.ndarray:
    """Noise-free unblurred lensed image of an analytic source, [ny, nx]."""
    tx, ty = image_centres(geom)
    ox, oy = subpixel_offsets(nsub, geom.pix)
    rx = (tx[:, None] + ox[None, :]).ravel()
    ry = (ty[:, None] + oy[None, :]).ravel()
    bx, by = ray_trace(rx, ry, lens)
    sb = eval_source(comps, bx, by).reshape(geom.npix, nsub * nsub).mean(axis=1)
    return sb.reshape(geom.ny, geom.nx)


def observe(geom, lens, comps, psf, noise, snr: float = 20.0, mask=None) -> Problem:
    """Blurred lensed image plus noise scaled to S/N = snr; returns a Problem.

    ``noise`` is a unit-Gaussian draw of shape [ny, nx].
    """
    clean = convolve2d(lensed_image(geom, lens, comps), psf, mode="same")
    sigma_val = clean.max() / snr
    d = clean + sigma_val * np.asarray(noise).reshape(geom.ny, geom.nx)
    sigma = np.full((geom.ny, geom.nx), sigma_val)
    if mask is None:
        mask = np.ones((geom.ny, geom.nx), dtype=np.uint8)
    return Problem(geom, d, sigma, mask, np.asarray(psf, dtype=np.float64))
