"""Oracle: explicit lens, blur, weight and regularisation matrices (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

* L (Section 2.1 and 2.2): each image (sub-)pixel is traced to the source
  plane and takes the bilinear interpolation of the four surrounding source
  pixel centres (the TK04 scheme the paper adopts); with N_p sub-pixels per
  image pixel the row is the mean of the sub-pixel rows (Section 2.2).  Rays
  outside the grid of source centres get no intensity (Section 2.2).
* B (Section 2.2): linear convolution with the K x K PSF, zero outside the
  image ('same' size), i.e. what a zero-padded FFT convolution computes.
* W = diag(m / sigma^2) with m = user mask AND mapped (Eq. chi2 restricted
  to image pixels that map back to the source plane, Section 2.2).
* H (Eq. TKReg): identity, forward-difference gradient [Dx; Dy], or the
  5-point Laplacian, with zero source intensity beyond the grid.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .lens import ray_trace

REG_IDENTITY, REG_GRADIENT, REG_LAPLACIAN = 0, 1, 2


def image_centres(geom):
    """Pixel-centre coordinates (x fast, y slow), each flattened to [npix]."""
    xs = geom.cx + (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.pix
    ys = geom.cy + (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.pix
    tx, ty = np.meshgrid(xs, ys)
    return tx.ravel(), ty.ravel()


def subpixel_offsets(n: int, pix: float):
    """Offsets of an n x n sub-pixel grid from the pixel centre, [n*n] each."""
    o = ((np.arange(n) + 0.5) / n - 0.5) * pix
    ox, oy = np.meshgrid(o, o)
    return ox.ravel(), oy.ravel()


def source_cell(geom, bx, by):
    """Bilinear cell of source-plane points.

    Returns (mapped, ix0, iy0, u, v): the point is mapped when it lies inside
    the rectangle spanned by the first and last source-pixel centres on both
    axes; (ix0, iy0) is the lower-left centre of its cell (the last cell when
    the point sits on the last centre) and (u, v) in [0, 1] its fractional
    offsets in that cell.
    """
    hx = (geom.sxmax - geom.sxmin) / geom.sx
    hy = (geom.symax - geom.symin) / geom.sy
    fx = (np.asarray(bx) - (geom.sxmin + 0.5 * hx)) / hx
    fy = (np.asarray(by) - (geom.symin + 0.5 * hy)) / hy
    mapped = (fx >= 0) & (fx <= geom.sx - 1) & (fy >= 0) & (fy <= geom.sy - 1)
    ix0 = np.minimum(np.floor(np.where(mapped, fx, 0.0)), geom.sx - 2).astype(np.int64)
    iy0 = np.minimum(np.floor(np.where(mapped, fy, 0.0)), geom.sy - 2).astype(np.int64)
    u = np.where(mapped, fx - ix0, 0.0)
    v = np.where(mapped, fy - iy0, 0.0)
    return mapped, ix0, iy0, u, v


INTERP_NEAREST = 1  # geometry.interp: all of a ray's weight on the nearest centre (WD03)
INTERP_BICUBIC = 2  # geometry.interp: Keys' cubic convolution over the 4 x 4 nearby centres

KEYS_A = -0.5  # the cubic-convolution parameter that makes the interpolant third-order accurate


def keys_kernel(t):
    """Keys' cubic-convolution kernel W(t) (Keys 1981) with a = -1/2:
    (a+2)|t|^3 - (a+3)|t|^2 + 1 for |t| <= 1, a|t|^3 - 5a|t|^2 + 8a|t| - 4a
    for 1 < |t| < 2, and 0 beyond."""
    a = KEYS_A
    t = np.abs(np.asarray(t, dtype=np.float64))
    inner = (a + 2) * t ** 3 - (a + 3) * t ** 2 + 1
    outer = a * t ** 3 - 5 * a * t ** 2 + 8 * a * t - 4 * a
    return np.where(t <= 1, inner, np.where(t < 2, outer, 0.0))


def nearest_centre(geom, ix0, iy0, u, v):
    """Nearest source-pixel centre of points in cell (ix0, iy0) at offsets
    (u, v): the upper centre of an axis once the offset reaches half a cell."""
    return ix0 + (u >= 0.5), iy0 + (v >= 0.5)


def lens_matrix(geom, lens):
    """Explicit lens operator L as CSR [npix, ns] and the per-pixel mapped flag.

    Bilinear (TK04): each mapped ray spreads 1/N_p over the four centres of
    its cell with weights (1-u)(1-v), u(1-v), (1-u)v, uv.  Nearest neighbour
    (geometry.interp == 1, WD03): each mapped ray puts 1/N_p on its nearest
    centre.  Bicubic (geometry.interp == 2, Section 2.1): each mapped ray
    puts 1/N_p W(dx) W(dy) on every centre, dx and dy its distances to the
    centre in cell widths and W Keys' kernel, so only the 4 x 4 centres
    around its cell get weight; centres beyond the grid do not exist, so
    their share is dropped.  A pixel is mapped when at least one of its
    sub-pixel rays is.
    """
    tx, ty = image_centres(geom)
    ox, oy = subpixel_offsets(geom.subpix, geom.pix)
    npix, ns, npsub = geom.npix, geom.ns, geom.subpix * geom.subpix
    # rays: pixel-major, sub-pixel minor
    rx = (tx[:, None] + ox[None, :]).ravel()
    ry = (ty[:, None] + oy[None, :]).ravel()
    bx, by = ray_trace(rx, ry, lens)
    mapped, ix0, iy0, u, v = source_cell(geom, bx, by)
    pix_of_ray = np.repeat(np.arange(npix), npsub)
    if getattr(geom, "interp", 0) == INTERP_NEAREST:
        jx, jy = nearest_centre(geom, ix0, iy0, u, v)
        L = sp.csr_matrix((np.full(int(mapped.sum()), 1.0 / npsub),
                           (pix_of_ray[mapped], (jy * geom.sx + jx)[mapped])), shape=(npix, ns))
        L.sum_duplicates()
        return L, mapped.reshape(npix, npsub).any(axis=1)
    rows, cols, vals = [], [], []
    if getattr(geom, "interp", 0) == INTERP_BICUBIC:
        fx, fy = ix0 + u, iy0 + v  # ray position in centre units
        for jy in range(-1, 3):
            for jx in range(-1, 3):
                cx, cy = ix0 + jx, iy0 + jy
                ok = mapped & (cx >= 0) & (cx < geom.sx) & (cy >= 0) & (cy < geom.sy)
                rows.append(pix_of_ray[ok])
                cols.append((cy * geom.sx + cx)[ok])
                vals.append((keys_kernel(fx - cx) * keys_kernel(fy - cy))[ok] / npsub)
        L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(npix, ns))
        L.sum_duplicates()
        return L, mapped.reshape(npix, npsub).any(axis=1)
    for dx, dy, w in ((0, 0, (1 - u) * (1 - v)), (1, 0, u * (1 - v)),
                      (0, 1, (1 - u) * v), (1, 1, u * v)):
        rows.append(pix_of_ray[mapped])
        cols.append(((iy0 + dy) * geom.sx + (ix0 + dx))[mapped])
        vals.append(w[mapped] / npsub)
    L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(npix, ns))
    L.sum_duplicates()
    pmapped = mapped.reshape(npix, npsub).any(axis=1)
    return L, pmapped


def blur_matrix(geom, psf, dense=None):
    """Explicit blur operator B [npix, npix]: (B x)[p] = sum_k psf[k] x[p - (k - c)].

    Dense for images up to 64x64, CSR above (same matrix).
    """
    psf = np.asarray(psf, dtype=np.float64)
    k = psf.shape[0]
    c = (k - 1) // 2
    nx, ny = geom.nx, geom.ny
    rows, cols, vals = [], [], []
    py, px = np.mgrid[0:ny, 0:nx]
    for ky in range(k):
        for kx in range(k):
            qy = py - (ky - c)
            qx = px - (kx - c)
            ok = (qy >= 0) & (qy < ny) & (qx >= 0) & (qx < nx)
            rows.append((py * nx + px)[ok])
            cols.append((qy * nx + qx)[ok])
            vals.append(np.full(int(ok.sum()), psf[ky, kx]))
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny))
    if dense is None:
        dense = nx * ny <= 4096
    return B.toarray() if dense else B


def weight_vector(mask, mapped, sigma):
    """Diagonal of W: m / sigma^2 with m = user mask AND mapped."""
    m = (np.asarray(mask).ravel() != 0) & np.asarray(mapped).ravel()
    return np.where(m, 1.0 / np.asarray(sigma, dtype=np.float64).ravel() ** 2, 0.0)


def reg_matrix(geom, reg):
    """Explicit regularisation operator H (CSR) on the sx x sy source grid."""
    sx, sy, ns = geom.sx, geom.sy, geom.ns
    if reg == REG_IDENTITY:
        return sp.identity(ns, format="csr")
    idx = np.arange(ns).reshape(sy, sx)
    if reg == REG_GRADIENT:
        # (Dx s)[j, i] = s[j, i+1] - s[j, i]; s beyond the last column is 0.
        Dx = sp.lil_matrix((ns, ns))
        Dy = sp.lil_matrix((ns, ns))
        for j in range(sy):
            for i in range(sx):
                r = idx[j, i]
                Dx[r, r] = -1.0
                if i + 1 < sx:
                    Dx[r, idx[j, i + 1]] = 1.0
                Dy[r, r] = -1.0
                if j + 1 < sy:
                    Dy[r, idx[j + 1, i]] = 1.0
        return sp.vstack([Dx.tocsr(), Dy.tocsr()]).tocsr()
    if reg == REG_LAPLACIAN:
        # (H s)[j, i] = 4 s[j, i] - sum of the four neighbours (missing = 0).
        Hm = sp.lil_matrix((ns, ns))
        for j in range(sy):
            for i in range(sx):
                r = idx[j, i]
                Hm[r, r] = 4.0
                for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                    jj, ii = j + dj, i + di
                    if 0 <= jj < sy and 0 <= ii < sx:
                        Hm[r, idx[jj, ii]] = -1.0
        return Hm.tocsr()
    raise ValueError(f"unknown regulariser {reg}")
