"""GPU parity of the blur engines (mirage_psf_blur) against the oracle's
explicit blur operator B (Section 2.2).

The FFMA engine (the CG kernel's register tiles) must agree to FP32
accumulation accuracy; the tensor-core engine (TF32 block-Toeplitz products
on tcgen05) within the TF32 rounding bound: each factor rounded to nearest
TF32 is within 2^-11 relative, so one application errs by at most about
2^-10 of sum |psf| |x| per output, and a stored intermediate adds 2^-11.
The PSF is non-negative (a normalised blur, like the paper's Gaussians), so
|B| = B and B^r |x| bounds the magnitudes of r applications.
"""
import numpy as np
import pytest
import torch

import synth
from oracle.operators import blur_matrix
from synth import Geometry, REG_LAPLACIAN

pytestmark = pytest.mark.gpu

K = 9


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding as b
    return b


def _geom(nx, ny):
    return Geometry(nx, ny, 0.05, 8, 8, -1.0, 1.0, -1.0, 1.0, K, 1, REG_LAPLACIAN)


def _apply(B, x, reps):
    for _ in range(reps):
        x = B @ x
    return x


# the workload's 64 x 64 image; one tensor-core tile (16 x 7, 32 x 20, 48 x 33:
# ragged strips and rows); several tiles with a ragged last one (48 x 96)
@pytest.mark.parametrize("nx,ny", [(64, 64), (16, 7), (32, 20), (48, 33), (48, 96)])
@pytest.mark.parametrize("reps", [1, 2])
def test_blur_engines_match_oracle(binding, nx, ny, reps):
    rng = np.random.default_rng(1000 * nx + 10 * ny + reps)
    n = 5
    imgs = rng.standard_normal((n, ny, nx)).astype(np.float32)
    psf = rng.uniform(0.0, 1.0, (K, K)).astype(np.float32)
    psf /= psf.sum()
    B = blur_matrix(_geom(nx, ny), psf.astype(np.float64), dense=True)
    X = imgs.reshape(n, -1).astype(np.float64).T
    ref = _apply(B, X, reps)
    mag = _apply(B, np.abs(X), reps)
    x = torch.as_tensor(imgs, device="cuda")
    o_f = binding.mirage_psf_blur(binding.MIRAGE_BLUR_FFMA, x, psf, reps).cpu().numpy().reshape(n, -1).T
    o_t = binding.mirage_psf_blur(binding.MIRAGE_BLUR_TC_TF32, x, psf, reps).cpu().numpy().reshape(n, -1).T
    bound_f = reps * (K * K + 2) * 2.0 ** -23 * mag + 1e-30
    assert np.all(np.abs(o_f - ref) <= bound_f), np.max(np.abs(o_f - ref) / bound_f)
    bound_t = ((2 * reps + 1) * 2.0 ** -11 + 1e-5) * mag + 1e-30
    assert np.all(np.abs(o_t - ref) <= bound_t), np.max(np.abs(o_t - ref) / bound_t)
    # the tensor-core result is not the FFMA one (TF32 factors): the bound is
    # not met through a copy of the other engine's output
    assert np.abs(o_t - o_f).max() > 0


def test_blur_engines_many_images(binding):
    """More images than resident CTAs: each CTA loops over several images and
    reuses its shared-memory buffers and tensor memory; sampled images are
    checked against the oracle with the workload's Gaussian PSF."""
    g = synth.geom_ga64()
    psf = synth.gaussian_psf(K, synth.PSF_SIGMA["ga64"]).astype(np.float32)
    n = 1500
    rng = np.random.default_rng(7)
    imgs = torch.as_tensor(rng.standard_normal((n, g.ny, g.nx)).astype(np.float32), device="cuda")
    B = blur_matrix(_geom(g.nx, g.ny), psf.astype(np.float64), dense=True)
    pick = [0, 1, 303, 304, 305, 607, 608, 911, 1215, 1499]
    X = imgs[pick].reshape(len(pick), -1).double().cpu().numpy().T
    ref, mag = B @ X, B @ np.abs(X)
    for eng, coef in ((binding.MIRAGE_BLUR_FFMA, (K * K + 2) * 2.0 ** -23),
                      (binding.MIRAGE_BLUR_TC_TF32, 3 * 2.0 ** -11 + 1e-5)):
        o = binding.mirage_psf_blur(eng, imgs, psf, 1)
        assert torch.isfinite(o).all()
        got = o[pick].reshape(len(pick), -1).double().cpu().numpy().T
        assert np.all(np.abs(got - ref) <= coef * mag + 1e-30), eng


def test_blur_rejects_unsupported_shapes(binding):
    x = torch.zeros((1, 16, 24), device="cuda")
    with pytest.raises(binding.MirageError, match="multiple of 16"):
        binding.mirage_psf_blur(binding.MIRAGE_BLUR_TC_TF32, x, np.ones((K, K)), 1)
    with pytest.raises(binding.MirageError, match="K must be 9"):
        binding.mirage_psf_blur(binding.MIRAGE_BLUR_FFMA, torch.zeros((1, 16, 16), device="cuda"),
                                np.ones((7, 7)), 1)
