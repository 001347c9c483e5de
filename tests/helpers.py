"""Shared test helpers: oracle problems -> device tensors, tolerance checks."""
from __future__ import annotations

import numpy as np
import torch

import synth
from oracle.data import observe
from oracle.solve import Problem


def device_problem(prob: Problem, dtype=torch.float32, device="cuda"):
    """Binding Problem with the oracle problem's arrays on the device."""
    from paper_1101_5803_gb300.binding import Problem as BP
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
    return BP(prob.geom, t(prob.d.ravel(), dtype), t(prob.sigma.ravel(), dtype),
              t(prob.mask.ravel(), torch.uint8), t(prob.psf.ravel(), dtype))


def host_problem(prob: Problem, dtype=torch.float32):
    return device_problem(prob, dtype, device="cpu")


def make_problem(geom, seed=0, psf_sigma=1.5, lens=synth.TRUE_LENS, mask=None, fixed_source=False):
    """Synthetic observation through the oracle (S/N 20, 4x4 sub-pixel data).

    The image, noise map and PSF are rounded to float32 values, so that the
    FP32 library and the FP64 oracle are handed the very same problem."""
    rng = np.random.default_rng(seed)
    comps = synth.two_gaussian_source() if fixed_source else synth.drawn_source(rng)
    psf = synth.gaussian_psf(geom.kpsf, psf_sigma)
    prob = observe(geom, lens, comps, psf, synth.standard_normal(rng, (geom.ny, geom.nx)), mask=mask)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return Problem(prob.geom, f32(prob.d), f32(prob.sigma), prob.mask, f32(prob.psf))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
