"""The autotuner picks a kernel variant per shape class, caches it, and
every variant it chooses between gives the same results (variants 1-3
bitwise, the general kernel within the parity tolerances)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_tune_caches_and_variants_agree(tmp_path, monkeypatch):
    monkeypatch.setenv("MIRAGE_TUNE_CACHE", str(tmp_path / "tune.json"))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import autotune, binding
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, 16, 4, seed=9)
    v = autotune.tune(ctx, [wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, n_probe=8)
    assert v in autotune.VARIANTS
    assert (tmp_path / "tune.json").exists()
    assert autotune.tune(ctx, [wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam) == v
    outs = {k: ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, variant=k)
            for k in autotune.VARIANTS}
    for k in (2, 3):
        assert torch.equal(outs[k]["chi2"], outs[1]["chi2"])
    # the general kernel solves the same systems to the same tolerance;
    # two solves to rel-res 1e-6 of systems with kappa ~ 1e7 differ in chi2
    # by up to ~1e-5 (the oracle-based gates live in test_gpu_parity)
    c1, c4 = outs[1]["chi2"].cpu().numpy(), outs[4]["chi2"].cpu().numpy()
    assert np.abs(c4 / c1 - 1).max() < 1e-4
    ctx.close()


def test_ffma_microbenchmark():
    # the FP32 FMA pipe sustains a large share of its nominal 256 flops per
    # clock per SM (the binding roof of the CGLS kernels), and never more
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    tf, fc = binding.mirage_measure_ffma(0)
    assert 0.3 * 256 < fc < 1.05 * 256, fc
    assert tf > 0


def test_tune_config_caches_and_agrees(tmp_path, monkeypatch):
    # the tuned (variant, inner target, placement) solves the same systems:
    # chi2 within the solver tolerance of the default configuration, and
    # the cached choice is returned on the next call
    monkeypatch.setenv("MIRAGE_TUNE_CACHE", str(tmp_path / "tune.json"))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import autotune, binding
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, 16, 6, seed=9)
    cfg = autotune.tune_config(ctx, [wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, n_probe=8, reps=1)
    assert cfg["variant"] in autotune.VARIANTS and cfg["inner_eta"] in autotune.ETAS
    assert cfg["place"] in (0,) + autotune.PLACES
    assert autotune.tune_config(ctx, [wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam) == cfg
    a = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, **cfg)
    b = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6)
    assert ((a["item_status"] & 7) == 0).all() and ((b["item_status"] & 7) == 0).all()
    c1, c2 = a["chi2"].cpu().numpy(), b["chi2"].cpu().numpy()
    assert np.abs(c1 / c2 - 1).max() < 1e-4
    ctx.close()


def test_general_kernel_placements_agree_bitwise():
    # the general kernel's work buffers in shared memory, split, or all in
    # the L2-resident slab (the last two with one or two CTAs per SM): the
    # same arithmetic in the same order
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import observe_on_device

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    g = synth.Geometry(48, 48, 6.4 / 48, 16, 16, -0.8, 0.8, -0.8, 0.8, 7, 1, synth.REG_LAPLACIAN)
    rng = np.random.default_rng(2)
    prob = observe_on_device(ctx, g, synth.gaussian_psf(7, 7 / 6), synth.drawn_source(rng), synth.TRUE_LENS, rng)
    lens = torch.as_tensor(synth.lens_population(rng, 6), device="cuda")
    lams = torch.as_tensor(np.tile(synth.lambda_grid(5), (6, 1)), device="cuda")
    outs = [ctx.eval_batch([prob], lens, [0] * 6, lams, [5] * 6, tol=1e-6, variant=4, place=p, want_all_x=True)
            for p in (1, 2, 3, 4, 5)]
    for o in outs[1:]:
        for key in ("chi2", "reg", "iters", "all_x"):
            assert torch.equal(o[key], outs[0][key]), key
    with pytest.raises(binding.MirageError):
        ctx.eval_batch([prob], lens, [0] * 6, lams, [5] * 6, place=7)
    ctx.close()


def test_tf32_precision_variant_reaches_the_same_solutions():
    # variant 7 rounds both factors of the inner solves' convolution products
    # to TF32 (the arithmetic of a TF32 tensor-core B/B^T); the FP64
    # refinement's residual stays exact, so every item still converges to the
    # same solution (chi2 within the solver tolerance of the FP32 variant)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, 24, 16, seed=4)
    a = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, variant=2)
    b = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, variant=7)
    assert ((a["item_status"] & 7) == 0).all()
    assert ((b["item_status"] & 7) == 0).all()
    assert (b["relres"] <= 1e-6).all()
    c1, c2 = a["chi2"].cpu().numpy(), b["chi2"].cpu().numpy()
    assert np.abs(c2 / c1 - 1).max() < 1e-4
    # the rounding changes the iteration path, so the counts differ
    assert not torch.equal(a["iters"], b["iters"])
    ctx.close()
