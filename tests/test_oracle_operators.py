"""Pins for the oracle's explicit operators L, B, W, H (Sections 2.1, 2.2).

L is pinned by exact reproduction of bilinear functions, the identity lens,
partition of unity and brute force on a tiny grid; B by SciPy's 2-D
convolution / correlation and the delta PSF; H by hand-computed stencils.
"""
import math

import numpy as np
import pytest
from scipy.signal import convolve2d, correlate2d

from oracle.lens import ray_trace
from oracle.operators import (REG_GRADIENT, REG_IDENTITY, REG_LAPLACIAN, blur_matrix, image_centres,
                              lens_matrix, reg_matrix, source_cell, weight_vector)
import synth
from synth import Geometry, gaussian_psf

LENS = [1.0, 0.7, 0.5, 0.02, -0.03, 0.05, 1.0]


def _geom(**kw):
    base = dict(nx=24, ny=20, pix=0.1, sx=12, sy=10, sxmin=-0.8, sxmax=0.8, symin=-0.7, symax=0.7,
                kpsf=5, subpix=1, reg=REG_LAPLACIAN)
    base.update(kw)
    return Geometry(**base)


def _source_centres(g):
    hx = (g.sxmax - g.sxmin) / g.sx
    hy = (g.symax - g.symin) / g.sy
    cx = g.sxmin + (np.arange(g.sx) + 0.5) * hx
    cy = g.symin + (np.arange(g.sy) + 0.5) * hy
    X, Y = np.meshgrid(cx, cy)
    return X.ravel(), Y.ravel()


@pytest.mark.parametrize("subpix", [1, 2, 3])
def test_bilinear_reproduces_bilinear_functions(subpix):
    g = _geom(subpix=subpix)
    L, mapped = lens_matrix(g, LENS)
    X, Y = _source_centres(g)
    f = lambda x, y: 0.3 + 1.7 * x - 0.4 * y + 2.1 * x * y
    model = L @ f(X, Y)
    # expected: mean over the mapped sub-rays of f(beta) (unmapped rays give 0)
    tx, ty = image_centres(g)
    o = ((np.arange(subpix) + 0.5) / subpix - 0.5) * g.pix
    ox, oy = np.meshgrid(o, o)
    rx = (tx[:, None] + ox.ravel()[None, :])
    ry = (ty[:, None] + oy.ravel()[None, :])
    bx, by = ray_trace(rx.ravel(), ry.ravel(), LENS)
    m, *_ = source_cell(g, bx, by)
    exp = np.where(m, f(bx, by), 0.0).reshape(g.npix, -1).mean(axis=1)
    np.testing.assert_allclose(model, exp, atol=1e-12)
    assert mapped.sum() > 0.3 * g.npix


def test_partition_of_unity_and_positivity():
    g = _geom()
    L, mapped = lens_matrix(g, LENS)
    rs = np.asarray(L.sum(axis=1)).ravel()
    np.testing.assert_allclose(rs[mapped], 1.0, atol=1e-13)
    assert np.all(rs[~mapped] == 0.0)
    assert L.data.min() >= 0.0


def test_identity_lens():
    # b = 0, no shear, source centres on the image centres: L = I
    g = Geometry(nx=8, ny=6, pix=0.1, sx=8, sy=6, sxmin=-0.4, sxmax=0.4, symin=-0.3, symax=0.3,
                 kpsf=3, subpix=1, reg=REG_IDENTITY)
    L, mapped = lens_matrix(g, [0.0, 0.8, 0.0, 0, 0, 0, 0])
    np.testing.assert_allclose(L.toarray(), np.eye(48), atol=1e-12)
    assert mapped.all()


def test_brute_force_tiny():
    # a 2x2 source and a 3x1 image, traced by hand through a pure shift
    # (b = 0, shear only would be linear; use the identity lens with an
    # offset source grid instead)
    g = Geometry(nx=3, ny=1, pix=0.5, sx=2, sy=2, sxmin=-0.5, sxmax=0.5, symin=-0.5, symax=0.5,
                 kpsf=1, subpix=1, reg=REG_IDENTITY)
    L, mapped = lens_matrix(g, [0.0, 0.8, 0.0, 0, 0, 0, 0])
    # source centres at +-0.25; image centres at x = -0.5, 0, 0.5, y = 0
    # x = 0 lies midway between the centres on both axes: weights 1/4 each
    Ld = L.toarray()
    assert list(mapped) == [False, True, False]
    np.testing.assert_allclose(Ld[1], [0.25, 0.25, 0.25, 0.25])
    np.testing.assert_allclose(Ld[0], 0.0)


def test_tie_on_last_centre():
    # unit cells, centres at -1.5, -0.5, 0.5, 1.5 (exact in binary)
    g = Geometry(nx=1, ny=1, pix=1.0, sx=4, sy=4, sxmin=-2.0, sxmax=2.0, symin=-2.0, symax=2.0,
                 kpsf=1, subpix=1, reg=REG_IDENTITY)
    m, ix, iy, u, v = source_cell(g, np.array([1.5]), np.array([1.5]))
    assert m[0] and ix[0] == 2 and iy[0] == 2 and u[0] == 1.0 and v[0] == 1.0
    m, ix, iy, u, v = source_cell(g, np.array([-1.5]), np.array([0.25]))
    assert m[0] and ix[0] == 0 and iy[0] == 1 and u[0] == 0.0 and v[0] == 0.75
    m, *_ = source_cell(g, np.array([1.5000001]), np.array([0.0]))
    assert not m[0]
    m, *_ = source_cell(g, np.array([0.0]), np.array([-1.5000001]))
    assert not m[0]


@pytest.mark.parametrize("k", [1, 3, 5, 9])
def test_blur_matches_scipy(k):
    g = _geom(kpsf=k)
    rng = np.random.default_rng(4)
    psf = rng.uniform(0, 1, (k, k))
    x = rng.standard_normal((g.ny, g.nx))
    y = rng.standard_normal((g.ny, g.nx))
    B = blur_matrix(g, psf)
    np.testing.assert_allclose((B @ x.ravel()).reshape(g.ny, g.nx), convolve2d(x, psf, mode="same"),
                               atol=1e-12)
    np.testing.assert_allclose((B.T @ y.ravel()).reshape(g.ny, g.nx), correlate2d(y, psf, mode="same"),
                               atol=1e-12)
    Bs = blur_matrix(g, psf, dense=False)
    np.testing.assert_allclose(Bs.toarray(), B, atol=0)


def test_delta_psf_is_identity():
    g = _geom(kpsf=5)
    psf = np.zeros((5, 5))
    psf[2, 2] = 1.0
    np.testing.assert_array_equal(blur_matrix(g, psf), np.eye(g.npix))


def test_gaussian_psf_normalised():
    p = gaussian_psf(9, 1.5)
    assert abs(p.sum() - 1.0) < 1e-14
    assert p[4, 4] == p.max()
    np.testing.assert_allclose(p, p.T)
    np.testing.assert_allclose(p, p[::-1, ::-1])


def test_weights():
    mask = np.array([[1, 1, 0]], dtype=np.uint8)
    mapped = np.array([True, False, True])
    sigma = np.array([[2.0, 2.0, 2.0]])
    np.testing.assert_allclose(weight_vector(mask, mapped, sigma), [0.25, 0.0, 0.0])


def test_regularisers_by_hand():
    g = Geometry(nx=1, ny=1, pix=1, sx=3, sy=2, sxmin=0, sxmax=3, symin=0, symax=2, kpsf=1)
    s = np.array([1.0, 2.0, 4.0, 0.5, -1.0, 3.0])  # rows: [1 2 4], [0.5 -1 3]
    np.testing.assert_allclose(reg_matrix(g, REG_IDENTITY) @ s, s)
    # gradient: Dx then Dy, zero beyond the grid
    dx = [2 - 1, 4 - 2, 0 - 4, -1 - 0.5, 3 + 1, 0 - 3]
    dy = [0.5 - 1, -1 - 2, 3 - 4, 0 - 0.5, 0 + 1, 0 - 3]
    np.testing.assert_allclose(reg_matrix(g, REG_GRADIENT) @ s, dx + dy)
    # Laplacian: 4 s - neighbours
    lap = [4 * 1 - 2 - 0.5, 4 * 2 - 1 - 4 + 1, 4 * 4 - 2 - 3,
           4 * 0.5 - 1 + 1, 4 * -1 - 0.5 - 3 - 2, 4 * 3 + 1 - 4]
    np.testing.assert_allclose(reg_matrix(g, REG_LAPLACIAN) @ s, lap)


@pytest.mark.parametrize("reg", [REG_IDENTITY, REG_GRADIENT, REG_LAPLACIAN])
def test_hth_positive_definite(reg):
    g = _geom()
    H = reg_matrix(g, reg).toarray()
    ev = np.linalg.eigvalsh(H.T @ H)
    assert ev.min() > 1e-6


def test_nearest_neighbour_lens_matrix_against_brute_force():
    # every mapped ray's whole weight sits on the closest source-pixel centre
    # (brute-force distance to all centres); unmapped rays get nothing
    import dataclasses
    from oracle.lens import ray_trace
    from oracle.operators import image_centres, lens_matrix, source_cell
    g = dataclasses.replace(synth.Geometry(20, 18, 0.09, 9, 8, -0.8, 0.8, -0.7, 0.7, 3, 1, synth.REG_IDENTITY),
                            interp=synth.INTERP_NEAREST)
    lens = [1.0, 0.7, 0.5, 0.02, -0.01, 0.05, 1.0]
    L, mapped = lens_matrix(g, lens)
    L = L.toarray()
    tx, ty = image_centres(g)
    bx, by = ray_trace(tx, ty, lens)
    m, *_ = source_cell(g, bx, by)
    hx, hy = (g.sxmax - g.sxmin) / g.sx, (g.symax - g.symin) / g.sy
    cxs = g.sxmin + (np.arange(g.sx) + 0.5) * hx
    cys = g.symin + (np.arange(g.sy) + 0.5) * hy
    for j in range(g.npix):
        if not m[j]:
            assert not L[j].any()
            continue
        d2 = (cxs[None, :] - bx[j]) ** 2 + (cys[:, None] - by[j]) ** 2
        k = int(np.argmin(d2))
        assert L[j, k] == 1.0 and L[j].sum() == 1.0, j
    assert m.sum() > 50


def test_nearest_neighbour_identity_lens():
    # centres on the pixel centres and no deflection: L = I
    import dataclasses
    from oracle.operators import lens_matrix
    g = dataclasses.replace(synth.Geometry(12, 8, 0.25, 12, 8, -1.5, 1.5, -1.0, 1.0, 3, 1, synth.REG_IDENTITY),
                            interp=synth.INTERP_NEAREST)
    L, mapped = lens_matrix(g, [0, 0.8, 0, 0, 0, 0, 0])
    np.testing.assert_allclose(L.toarray(), np.eye(96), atol=0)
    assert mapped.all()


# ---------------------------------------------------------------------------
# bicubic interpolation (Keys' cubic convolution, a = -1/2)
# ---------------------------------------------------------------------------
def test_keys_kernel_is_an_interpolating_c1_cubic():
    from oracle.operators import keys_kernel
    # interpolating: 1 at the own centre, 0 at every other centre
    np.testing.assert_array_equal(keys_kernel([0.0, 1.0, -1.0, 2.0, -2.0, 3.0]), [1, 0, 0, 0, 0, 0])
    t = np.linspace(-2.5, 2.5, 1001)
    np.testing.assert_allclose(keys_kernel(t), keys_kernel(-t), atol=0)
    assert np.all(keys_kernel(t[np.abs(t) >= 2]) == 0)
    # continuous with a continuous slope at the knots |t| = 1, 2
    h = 1e-7
    for k in (1.0, 2.0):
        left, right = keys_kernel(k - h), keys_kernel(k + h)
        assert abs(left - right) < 1e-6
        dl = (keys_kernel(k - h) - keys_kernel(k - 2 * h)) / h
        dr = (keys_kernel(k + 2 * h) - keys_kernel(k + h)) / h
        assert abs(dl - dr) < 1e-5, (k, dl, dr)


def test_keys_weights_reproduce_quadratics_and_the_midpoint_rule():
    # sum_j W(u - j) j^m = u^m for m = 0, 1, 2 (the kernel's third-order
    # accuracy, Keys 1981); a cubic is not reproduced
    from oracle.operators import keys_kernel
    j = np.arange(-1, 3)
    for u in np.linspace(0, 1, 13):
        w = keys_kernel(u - j)
        for m in range(3):
            assert abs((w * j ** m).sum() - u ** m) < 1e-14, (u, m)
    w = keys_kernel(0.3 - j)
    assert abs((w * j ** 3).sum() - 0.3 ** 3) > 1e-3
    # halfway between two centres: the four-point rule (-1, 9, 9, -1)/16
    np.testing.assert_allclose(keys_kernel(0.5 - j), np.array([-1, 9, 9, -1]) / 16.0, atol=1e-15)


def _bicubic_geom(nx=20, ny=18, subpix=1):
    import dataclasses
    return dataclasses.replace(synth.Geometry(nx, ny, 0.09, 9, 8, -0.8, 0.8, -0.7, 0.7, 3, subpix, synth.REG_IDENTITY),
                               interp=synth.INTERP_BICUBIC)


def test_bicubic_lens_matrix_against_brute_force():
    # every centre of the grid weighted by W(dx) W(dy) from the traced
    # position, without using the cell of the ray
    from oracle.lens import ray_trace
    from oracle.operators import image_centres, keys_kernel, lens_matrix, source_cell
    g = _bicubic_geom()
    lens = [1.0, 0.7, 0.5, 0.02, -0.01, 0.05, 1.0]
    L, mapped = lens_matrix(g, lens)
    L = L.toarray()
    tx, ty = image_centres(g)
    bx, by = ray_trace(tx, ty, lens)
    m, *_ = source_cell(g, bx, by)
    hx, hy = (g.sxmax - g.sxmin) / g.sx, (g.symax - g.symin) / g.sy
    cxs = g.sxmin + (np.arange(g.sx) + 0.5) * hx
    cys = g.symin + (np.arange(g.sy) + 0.5) * hy
    for j in range(g.npix):
        if not m[j]:
            assert not L[j].any()
            continue
        w = keys_kernel((cys[:, None] - by[j]) / hy) * keys_kernel((cxs[None, :] - bx[j]) / hx)
        np.testing.assert_allclose(L[j], w.ravel(), atol=1e-14)
    assert m.sum() > 50


def test_bicubic_lens_matrix_reproduces_biquadratic_sources():
    # s = f at the centres, f a product-space quadratic: L s = f at every ray
    # whose 4 x 4 centres all lie in the grid (bilinear would miss the curvature)
    from oracle.lens import ray_trace
    from oracle.operators import image_centres, lens_matrix, source_cell
    g = _bicubic_geom()
    lens = [1.0, 0.7, 0.5, 0.02, -0.01, 0.05, 1.0]
    L, _ = lens_matrix(g, lens)
    hx, hy = (g.sxmax - g.sxmin) / g.sx, (g.symax - g.symin) / g.sy
    cx = g.sxmin + (np.arange(g.sx) + 0.5) * hx
    cy = g.symin + (np.arange(g.sy) + 0.5) * hy

    def f(x, y):
        return 1 + 0.3 * x - 0.7 * y + 0.9 * x * x - 0.4 * x * y + 0.6 * y * y + 0.8 * x * x * y * y

    s = f(cx[None, :], cy[:, None]).ravel()
    tx, ty = image_centres(g)
    bx, by = ray_trace(tx, ty, lens)
    m, ix0, iy0, _, _ = source_cell(g, bx, by)
    inner = m & (ix0 >= 1) & (ix0 <= g.sx - 3) & (iy0 >= 1) & (iy0 <= g.sy - 3)
    assert inner.sum() > 20
    np.testing.assert_allclose((L @ s)[inner], f(bx, by)[inner], atol=1e-12)
    # the bilinear operator does not reproduce it
    import dataclasses
    Lb, _ = lens_matrix(dataclasses.replace(g, interp=synth.INTERP_BILINEAR), lens)
    assert np.abs((Lb @ s)[inner] - f(bx, by)[inner]).max() > 1e-4


def test_bicubic_identity_lens_and_subpixel_average():
    import dataclasses
    from oracle.operators import lens_matrix
    g = dataclasses.replace(synth.Geometry(12, 8, 0.25, 12, 8, -1.5, 1.5, -1.0, 1.0, 3, 1, synth.REG_IDENTITY),
                            interp=synth.INTERP_BICUBIC)
    L, mapped = lens_matrix(g, [0, 0.8, 0, 0, 0, 0, 0])
    np.testing.assert_allclose(L.toarray(), np.eye(96), atol=1e-15)
    assert mapped.all()
    # with 2 x 2 sub-pixels each row averages its rays: rows of interior
    # pixels (all four rays' centres in the grid) sum to one
    g2 = _bicubic_geom(subpix=2)
    L2, m2 = lens_matrix(g2, [1.0, 0.7, 0.5, 0.02, -0.01, 0.05, 1.0])
    rows = np.asarray(L2.sum(axis=1)).ravel()
    assert np.all(rows[~m2] == 0)
    assert np.isclose(rows[m2], 1.0, atol=1e-12).sum() > 0.5 * m2.sum()


# ---------------------------------------------------------------------------
# the FFT blur's grid bound (the reading behind the FFT convolution path)
# ---------------------------------------------------------------------------
def _fft_blur(img, psf, M, corr=False):
    """B img (or B^T img) as the crop of a circular convolution on an M x M
    grid with the PSF centred at (0, 0), by numpy's FFT."""
    ny, nx = img.shape
    K = psf.shape[0]
    c = (K - 1) // 2
    pc = np.zeros((M, M))
    for a in range(K):
        for b in range(K):
            pc[(a - c) % M, (b - c) % M] += psf[a, b]
    S = np.fft.fft2(pc)
    if corr:
        S = np.conj(S)
    X = np.zeros((M, M))
    X[:ny, :nx] = img
    return np.real(np.fft.ifft2(np.fft.fft2(X) * S))[:ny, :nx]


@pytest.mark.parametrize("ny,nx,K", [(12, 10, 5), (9, 14, 9), (8, 8, 17), (20, 7, 13)])
def test_fft_grid_bound_reproduces_the_zero_padded_blur(ny, nx, K):
    # M >= max(nx, ny) + (K - 1)/2 gives exactly the oracle's B and B^T (the
    # wrap of the centred PSF lands in the zero padding); one row or column
    # less and the wrap aliases into the image
    from oracle.operators import blur_matrix
    rng = np.random.default_rng(K)
    g = synth.Geometry(nx, ny, 0.1, 4, 4, -0.8, 0.8, -0.8, 0.8, K, 1, synth.REG_IDENTITY)
    psf = rng.random((K, K))
    B = blur_matrix(g, psf, dense=True)
    img = rng.standard_normal((ny, nx))
    M = max(nx, ny) + (K - 1) // 2
    np.testing.assert_allclose(_fft_blur(img, psf, M).ravel(), B @ img.ravel(), atol=1e-12)
    np.testing.assert_allclose(_fft_blur(img, psf, M, corr=True).ravel(), B.T @ img.ravel(), atol=1e-12)
    assert np.abs(_fft_blur(img, psf, M - 1).ravel() - B @ img.ravel()).max() > 1e-6
