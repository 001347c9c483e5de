"""GPU parity of the fixed-iteration CGLS (mirage_eval_iter: the paper's
iteration L-curve, Section 2.6, and Monte Carlo degrees of freedom, Section
2.5) against the FP64 oracle (oracle/iterlc.py).

Both sides compute in FP64.  Without a regulariser CGLS loses orthogonality
after a few iterations, and from then on two correct FP64 runs that add in
different orders drift apart (measured: 1e-15 agreement on chi^2 through
iteration 10, up to 1e-2 by iteration 40).  What is unique is the
exact-arithmetic trajectory, which both follow until then, so the gates are:

  * iterations 0..6: chi^2 to 1e-12 (FP64 context) or 1e-6 (FP32 context,
    whose sqrt(W) is rounded to float), sum s^2 to 1e-8 / 1e-7, dof to
    1e-7 / 1e-5 of the fitted-pixel count;
  * the corner iteration is the oracle's, and the returned source matches
    the oracle's iterate there to 1e-9 / 1e-6;
  * every iteration: finite records, chi^2 never rising, dof within
    (0, 1.5 N_fit].
"""
import numpy as np
import pytest
import torch

import synth
from oracle.iterlc import cgls_iterations

from .helpers import device_problem, make_problem
from .test_gpu_parity import ctx32, ctx64, mods  # noqa: F401 (fixtures)

pytestmark = pytest.mark.gpu

N_ITER = 40
K_STABLE = 6


def _run(ctx, geom, prob, lenses, bhat, dt):
    L = torch.as_tensor(np.asarray(lenses, dtype=np.float64).reshape(-1, 7), device="cuda")
    b = torch.as_tensor(bhat.ravel()[None, :], dtype=dt, device="cuda")
    return ctx.eval_iter([device_problem(prob, dt)], L, [0] * len(lenses), N_ITER, bhat=b)


def _check(out, prob, lenses, bhat, tol_chi, tol_reg, tol_dof, tol_s):
    ns = prob.geom.sx * prob.geom.sy
    for c, lens in enumerate(lenses):
        r = cgls_iterations(prob, lens, N_ITER, bhat=bhat)
        chi = out["chi2"][c].cpu().numpy()
        reg = out["reg"][c].cpu().numpy()
        dof = out["dof"][c].cpu().numpy()
        n_fit = r.dof[0]
        k = K_STABLE + 1
        assert np.all(np.abs(chi[:k] / r.chi2[:k] - 1) <= tol_chi), (c, chi[:k], r.chi2[:k])
        assert np.all(np.abs(reg[1:k] / r.reg[1:k] - 1) <= tol_reg), (c, reg[:k], r.reg[:k])
        assert np.all(np.abs(dof[:k] - r.dof[:k]) <= tol_dof * n_fit), (c, dof[:k], r.dof[:k])
        assert int(out["corner"][c]) == r.corner, (c, int(out["corner"][c]), r.corner)
        s = out["s"][c, :ns].double().cpu().numpy()
        xr = r.xs[r.corner]
        assert np.linalg.norm(s - xr) <= tol_s * np.linalg.norm(xr), c
        assert np.all(np.isfinite(chi)) and np.all(np.isfinite(reg)) and np.all(np.isfinite(dof))
        assert np.all(np.diff(chi) <= 1e-9 * chi[0]), c
        assert np.all((dof > 0) & (dof <= 1.5 * n_fit)), c
        assert int(out["status"][c]) == (32 if r.flat else 0)


def test_iter_lcurve_fp64(mods, ctx64):
    g = synth.geom_small_fp64()
    prob = make_problem(g, seed=21)
    rng = np.random.default_rng(3)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 3)])
    bhat = rng.standard_normal((g.ny, g.nx))
    out = _run(ctx64, g, prob, lenses, bhat, torch.float64)
    _check(out, prob, lenses, bhat, 1e-12, 1e-8, 1e-7, 1e-9)


def test_iter_lcurve_fp32_context_64px(mods, ctx32):
    g = synth.geom_ga64()
    prob = make_problem(g, seed=21)
    rng = np.random.default_rng(3)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 3)])
    bhat = rng.standard_normal((g.ny, g.nx))
    out = _run(ctx32, g, prob, lenses, bhat, torch.float32)
    _check(out, prob, lenses, bhat, 1e-6, 1e-7, 1e-5, 1e-6)


def test_iter_lcurve_statuses_and_arguments(mods, ctx32):
    g = synth.geom_ga64()
    prob = make_problem(g, seed=22)
    bad = synth.TRUE_LENS.copy()
    bad[1] = np.nan                      # BAD_PARAM: chi^2 = +inf
    far = synth.TRUE_LENS.copy()
    far[0] = 50.0                        # every ray deflected far off the source grid: EMPTY_MAP
    lenses = np.vstack([synth.TRUE_LENS, bad, far])
    L = torch.as_tensor(lenses, device="cuda")
    dp = device_problem(prob)
    out = ctx32.eval_iter([dp], L, [0, 0, 0], 12)
    st = out["status"].cpu().numpy()
    assert st[1] & 8 and np.isinf(out["chi2"][1].cpu().numpy()).all()
    assert st[2] & 16 and (out["chi2"][2].cpu().numpy() == 0).all()
    assert not (st[0] & 0x1f) and 1 <= int(out["corner"][0]) <= 12
    assert "dof" not in out
    with pytest.raises(mods.MirageError):
        ctx32.eval_iter([dp], L, [0, 0, 0], 0)
    with pytest.raises(mods.MirageError):
        ctx32.eval_iter([dp], L, [0, 0, 0], 64)
    with pytest.raises(mods.MirageError):  # bhat rows shorter than the image
        ctx32.eval_iter([dp], L, [0, 0, 0], 8, bhat=torch.zeros((1, 100), device="cuda"))


def test_split_ray_trace_matches_fused(mods, ctx32):
    # few candidates on a large image take the split ray trace (many CTAs per
    # candidate trace, one places); as many candidates as SMs take the fused
    # one.  Both place the rays in the same order: identical records.
    g = synth.Geometry(128, 128, 0.03, 48, 48, -0.8, 0.8, -0.8, 0.8, 11, 1, synth.REG_LAPLACIAN)
    prob = make_problem(g, seed=23, psf_sigma=1.5)
    dp = device_problem(prob)
    rng = np.random.default_rng(4)
    lenses = np.vstack([synth.TRUE_LENS, synth.lens_population(rng, 1)])
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    few = ctx32.eval_iter([dp], torch.as_tensor(lenses, device="cuda"), [0, 0], 12)
    many_l = np.vstack([lenses] * ((n_sm + 1) // 2 + 1))
    many = ctx32.eval_iter([dp], torch.as_tensor(many_l, device="cuda"), [0] * len(many_l), 12)
    for key in ("chi2", "reg", "corner", "s"):
        assert torch.equal(few[key][:2].cpu(), many[key][:2].cpu()), key
