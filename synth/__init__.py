"""Seeded synthetic inputs for the lens-inversion inner loop.

This module is shared by the CPU oracle (tests) and the GPU path (bench,
smoke).  It draws random numbers and lays out plain input arrays only: it
holds none of the method's arithmetic (no ray tracing, no interpolation, no
blurring, no solve).  Lensed data images are made by whichever side needs
them (the oracle in tests, the GPU forward model in the benchmark).

Workload shapes follow the paper's test problems (Section 2.3, 2.7, 4.1) as
restated in the five workloads below; every drawn quantity takes its numbers
from a ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Regulariser codes (Eq. TKReg with H = I, a forward-difference gradient or a
# 5-point Laplacian).
REG_IDENTITY, REG_GRADIENT, REG_LAPLACIAN = 0, 1, 2

# Source-plane interpolation codes (Section 2.1).
INTERP_BILINEAR, INTERP_NEAREST, INTERP_BICUBIC = 0, 1, 2

# Lens parameter vector: SIE (Eqs. SIEX/SIEY) plus external shear.
LENS_KEYS = ("b", "q", "phi", "x0", "y0", "gamma", "theta_g")


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Image grid, source grid, PSF size, sub-pixels and regulariser.

    Image pixel centres are ``cx + (i - (nx-1)/2) * pix`` (x fast) and
    ``cy + (j - (ny-1)/2) * pix``; arrays are row-major with y the slow axis.
    The source grid is given by its outer edges; its ``sx * sy`` pixel centres
    sit half a cell inside them.
    """

    nx: int
    ny: int
    pix: float
    sx: int
    sy: int
    sxmin: float
    sxmax: float
    symin: float
    symax: float
    kpsf: int
    subpix: int = 1
    reg: int = REG_LAPLACIAN
    cx: float = 0.0
    cy: float = 0.0
    interp: int = 0  # INTERP_BILINEAR, INTERP_NEAREST or INTERP_BICUBIC

    @property
    def npix(self) -> int:
        return self.nx * self.ny

    @property
    def ns(self) -> int:
        return self.sx * self.sy


def gaussian_psf(k: int, sigma_px: float) -> np.ndarray:
    """K x K Gaussian PSF sampled at integer pixel offsets, unit sum."""
    c = (k - 1) / 2.0
    y, x = np.mgrid[0:k, 0:k].astype(np.float64)
    p = np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2.0 * sigma_px ** 2))
    return p / p.sum()


def lambda_grid(n: int, lo: float = 1e-4, hi: float = 1e2) -> np.ndarray:
    """n values log-spaced over [lo, hi], ascending."""
    return np.logspace(math.log10(lo), math.log10(hi), n)


@dataclasses.dataclass(frozen=True)
class SourceComponent:
    """Elliptical Gaussian source component (amp, sigma, axis ratio, centre, angle)."""

    amp: float
    sigma: float
    q: float
    xc: float
    yc: float
    angle: float = 0.0


def two_gaussian_source() -> list[SourceComponent]:
    """The fixed two-component source of the 32x32 FP64 problem."""
    return [SourceComponent(1.0, 0.12, 0.8, 0.05, 0.02, 0.0),
            SourceComponent(0.5, 0.08, 0.6, -0.10, 0.08, 0.0)]


def drawn_source(rng: np.random.Generator, n: int = 2) -> list[SourceComponent]:
    """n elliptical Gaussians with amplitude, width, ratio, centre and angle drawn."""
    out = []
    for _ in range(n):
        out.append(SourceComponent(
            amp=float(rng.uniform(0.5, 1.0)), sigma=float(rng.uniform(0.06, 0.15)),
            q=float(rng.uniform(0.5, 1.0)), xc=float(rng.uniform(-0.15, 0.15)),
            yc=float(rng.uniform(-0.15, 0.15)), angle=float(rng.uniform(0.0, math.pi))))
    return out


def eval_source(comps, bx: np.ndarray, by: np.ndarray) -> np.ndarray:
    """Surface brightness of a sum of elliptical Gaussians at source-plane points."""
    out = np.zeros(np.broadcast(bx, by).shape)
    for c in comps:
        ca, sa = math.cos(c.angle), math.sin(c.angle)
        u = ca * (bx - c.xc) + sa * (by - c.yc)
        v = -sa * (bx - c.xc) + ca * (by - c.yc)
        out += c.amp * np.exp(-0.5 * ((u / c.sigma) ** 2 + (v / (c.q * c.sigma)) ** 2))
    return out


TRUE_LENS = np.array([1.0, 0.7, 0.5, 0.0, 0.0, 0.05, 1.0])

# Bounds of the GA search box (b, q, phi, x0, y0, gamma, theta_g).
LENS_LO = np.array([0.8, 0.5, 0.0, -0.1, -0.1, 0.0, 0.0])
LENS_HI = np.array([1.2, 1.0, math.pi, 0.1, 0.1, 0.1, math.pi])


def lens_population(rng: np.random.Generator, n: int) -> np.ndarray:
    """n candidate lens vectors drawn uniformly in the search box, ``[n, 7]``."""
    return rng.uniform(LENS_LO, LENS_HI, size=(n, 7))


def annular_mask(geom: Geometry, r_in: float, r_out: float) -> np.ndarray:
    """uint8 mask of image pixels whose centre radius is in [r_in, r_out]."""
    xs = geom.cx + (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.pix
    ys = geom.cy + (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.pix
    r = np.hypot(xs[None, :], ys[:, None])
    return ((r >= r_in) & (r <= r_out)).astype(np.uint8)


def standard_normal(rng: np.random.Generator, shape) -> np.ndarray:
    """Unit Gaussian noise draw (scaled by the caller to the chosen S/N)."""
    return rng.standard_normal(shape)


# --------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------

def geom_small_fp64() -> Geometry:
    """32x32 image at 0.1"/px, 16x16 source over +-0.8", 5x5 PSF, gradient H."""
    return Geometry(32, 32, 0.1, 16, 16, -0.8, 0.8, -0.8, 0.8, 5, 1, REG_GRADIENT)


def geom_ga64() -> Geometry:
    """64x64 image at 0.05"/px, 32x32 source over +-0.8", 9x9 PSF, Laplacian H."""
    return Geometry(64, 64, 0.05, 32, 32, -0.8, 0.8, -0.8, 0.8, 9, 1, REG_LAPLACIAN)


def geom_e2e128() -> Geometry:
    """128x128 image at 0.03"/px, 48x48 source over +-0.8", 11x11 PSF."""
    return Geometry(128, 128, 0.03, 48, 48, -0.8, 0.8, -0.8, 0.8, 11, 1, REG_LAPLACIAN)


def geom_large256() -> Geometry:
    """256x256 image at 0.02"/px, 128x128 source over +-1.2", 21x21 PSF."""
    return Geometry(256, 256, 0.02, 128, 128, -1.2, 1.2, -1.2, 1.2, 21, 1, REG_LAPLACIAN)


PSF_SIGMA = {"small_fp64": 1.0, "ga64": 1.5, "e2e128": 1.5, "large256": 3.0}


@dataclasses.dataclass
class UnevenItem:
    """One problem class of the uneven batch: geometry, PSF, mask radii, n_lambda."""

    geom: Geometry
    psf_sigma: float
    r_in: float
    r_out: float
    n_lam: int


def uneven_batch(rng: np.random.Generator, n: int) -> list[UnevenItem]:
    """n uneven problems: image {48,64,96,128}^2 over 6.4", annular masks,
    source {16,24,32,48}^2 over +-0.8", PSF width {7,11,15} (sigma = width/6),
    8..32 lambda values."""
    out = []
    for _ in range(n):
        nim = int(rng.choice([48, 64, 96, 128]))
        nsrc = int(rng.choice([16, 24, 32, 48]))
        k = int(rng.choice([7, 11, 15]))
        g = Geometry(nim, nim, 6.4 / nim, nsrc, nsrc, -0.8, 0.8, -0.8, 0.8, k, 1, REG_LAPLACIAN)
        out.append(UnevenItem(g, k / 6.0, float(rng.uniform(0.3, 0.6)),
                              float(rng.uniform(1.5, 2.5)), int(rng.integers(8, 33))))
    return out
