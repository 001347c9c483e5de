"""Benchmark: lens-model evaluations per second on the 64x64 GA workload.

One step = one batched evaluation of a 256-candidate population: ray trace,
CGLS to relative residual 1e-6 for each of 16 lambdas (log-spaced 1e-4..1e2,
Laplacian regulariser) and the L-curve corner of every candidate
(64x64 image at 0.05"/px, 32x32 source over +-0.8", 9x9 Gaussian PSF).

Prints one JSON line.  ``value`` is device-timed throughput with inputs
resident in HBM; ``e2e`` is the same metric through the C ABI with pinned
host buffers (copies inside the timed region); ``roofline`` is for the CGLS
kernel (FP32 FFMA pipe); ``cpu_baseline`` is the FP64 oracle on the host
cores on a bounded sample; ``plain`` is the one-candidate-per-launch
evaluator on a sample of the same population.

``--impl reference`` times the CPU oracle alone on the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lens-model evals/s at 64^2 image, CG rel-res 1e-6 (256 cand x 16 lambda)"
UNIT = "evals/s"
N_CAND, N_LAM, TOL = 256, 16, 1e-6
TIGHT_TOL = 2e-8  # the tighter internal tolerance of the accuracy section
CONFIG = {"workload": "ga64: 64x64 image 0.05\"/px, 32x32 source +-0.8\", 9x9 PSF sigma 1.5px, Laplacian H, "
                      "256 candidates x 16 lambdas 1e-4..1e2, CGLS rel-res 1e-6, L-curve corner",
          "global_batch": N_CAND, "n_lambda": N_LAM, "l2": "flushed between timed steps (512 MiB write)"}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def _cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_evals_per_s(n_sample: int, seed: int = 0, budget_s: float = 20.0):
    """The FP64 oracle (dense Cholesky per lambda + L-curve) on a sample of the workload."""
    import synth
    from oracle.data import observe
    from oracle.solve import eval_candidate
    rng = np.random.default_rng(seed)
    g = synth.geom_ga64()
    comps = synth.drawn_source(rng)
    prob = observe(g, synth.TRUE_LENS, comps, synth.gaussian_psf(9, 1.5), synth.standard_normal(rng, (64, 64)))
    pop = synth.lens_population(rng, n_sample)
    lams = synth.lambda_grid(N_LAM)
    t0 = time.perf_counter()
    done = 0
    for lens in pop:
        eval_candidate(prob, lens, lams)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def flops_per_item(geom, iters):
    """Algorithmic FLOPs of one CGLS item: iters x F_it + one chi2 forward pass.

    F_it = 4 K^2 N_pix (B and B^T) + 16 N_pix (L, L^T) + 20 N_s (Laplacian
    H^T H) + 12 N_s (vector updates and dots)."""
    npix, ns, k = geom.nx * geom.ny, geom.ns, geom.kpsf
    f_it = 4 * k * k * npix + 16 * npix + 20 * ns + 12 * ns
    return iters * f_it + (2 * k * k * npix + 6 * npix)


def max_over_ranks(t: float, world: int, device=None) -> float:
    """Largest per-rank time (the job's time under weak scaling)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank: int, steps: int, t_max: float, world: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / t_max


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return 0
    per_step = max(2, int(os.environ.get("MIRAGE_REF_SAMPLE", "4")))
    vals = []
    for s in range(args.warmup + args.steps):
        v, done, dt = oracle_evals_per_s(per_step, seed=s, budget_s=60.0)
        if s >= args.warmup:
            vals.append((v, done, dt))
    tot_done = sum(d for _, d, _ in vals)
    tot_t = sum(t for _, _, t in vals)
    value = tot_done / tot_t
    cores = _cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} candidates x {N_LAM} lambdas per step (dense Cholesky)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _guarded(name, fn):
    """Run one secondary section of the benchmark; an exception is recorded in
    the JSON line (and its traceback printed to stderr) instead of ending the
    run, so the headline measurement is always reported."""
    import traceback
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - report and continue
        traceback.print_exc()
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import ga64_workload

    ctx = binding.Context(local, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, N_CAND, N_LAM, seed=1000 + rank)
    probs = [wl.problem]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    from paper_1101_5803_gb300.autotune import tune_config
    tcfg = tune_config(ctx, probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=TOL)
    variant = tcfg["variant"]

    def step(out=None, graph=True, timing=False):
        return ctx.eval_batch(probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=TOL, use_graph=graph,
                              out=out, want_kappa=True, phase_timing=timing, **tcfg)

    # untimed: one phase-timed call for the kernel roofline, then graph warm-up
    out = step(graph=False, timing=True)
    torch.cuda.synchronize()
    phase = ctx.phase_ms()
    iters = out["iters"].cpu().numpy()
    relres = out["relres"].cpu().numpy()
    status = out["status"].cpu().numpy()
    item_status = out["item_status"].cpu().numpy()
    for _ in range(args.warmup):
        out = step(out=out)
    torch.cuda.synchronize()
    launches_per_step = ctx.launches()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(st)
            out = step(out=out)
            ev[i][1].record(st)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(times) / 1e3
    t_max = max_over_ranks(t_total, world, device="cuda")
    value = job_throughput(N_CAND, args.steps, t_max, world)

    # end to end through the C ABI with pinned host buffers
    hp = binding.Problem(wl.geom, wl.problem.d.cpu().pin_memory(), wl.problem.sigma.cpu().pin_memory(),
                         wl.problem.mask.cpu().pin_memory(), wl.problem.psf.cpu().pin_memory())
    hl = wl.lens.cpu().pin_memory()
    hlam = wl.lambdas.cpu().pin_memory()
    hout = ctx.eval_batch([hp], hl, wl.prob_idx, hlam, wl.n_lam, tol=TOL, **tcfg)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hout = ctx.eval_batch([hp], hl, wl.prob_idx, hlam, wl.n_lam, tol=TOL, out=hout, **tcfg)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    h2d = sum(t.numel() * t.element_size() for t in (hp.d, hp.sigma, hp.mask, hp.psf, hl, hlam))
    d2h = sum(t.numel() * t.element_size() for t in hout.values())

    # plain evaluator (one candidate per launch sequence) on a sample: one
    # warm-up call on two candidates, then a call timed with CUDA events on
    # the launching stream
    n_plain = int(os.environ.get("MIRAGE_PLAIN_SAMPLE", "32"))

    def plain_call(n):
        return ctx.eval_batch(probs, wl.lens[:n].contiguous(), wl.prob_idx[:n], wl.lambdas[:n].contiguous(),
                              wl.n_lam[:n], tol=TOL, mode=binding.MIRAGE_MODE_PLAIN, **tcfg)

    plain_call(2)
    torch.cuda.synchronize()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(st)
    pout = plain_call(n_plain)
    pe1.record(st)
    torch.cuda.synchronize()
    plain = n_plain / (pe0.elapsed_time(pe1) / 1e3)
    same = bool(torch.equal(pout["chi2"], out["chi2"][:n_plain]))

    # roofline of the CGLS kernel: algorithmic FLOPs / its event-timed duration
    flops = float(sum(flops_per_item(wl.geom, int(i)) for i in iters.ravel()))
    t_cgls = phase[1] / 1e3
    peaks, src = measured_peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    peak = nsm * 128 * 2 * smax * 1e6 / 1e12
    achieved = flops / t_cgls / 1e12
    clocks = clk.summary()
    at_clock = None
    if clocks.get("sm_mhz"):
        at_clock = nsm * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12
    # the FP32 FMA pipe's sustained rate, measured by the library's microbenchmark
    ffma_tf, ffma_fc = binding.mirage_measure_ffma(local)
    kernel_name = {1: "k_cgls_fast<9,4,smem taps FFMA2> (two CTAs/SM)",
                   2: "k_cgls_fast<9,4,param taps FFMA> (two CTAs/SM)",
                   3: "k_cgls_fast<9,4,param taps FFMA2> (two CTAs/SM)",
                   4: "k_cgls<float,9,smem> (one CTA/SM)"}.get(variant, "k_cgls_fast<9,4,*>")

    # DRAM bytes per launch: the per-item traffic of the ncu capture of this
    # kernel (profiles/k_cgls_fast_ga64.md) times the items of one launch
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "k_cgls_fast_ga64.md")
    if os.path.exists(tfile):
        for line in open(tfile):
            if line.startswith("traffic_bytes_per_item:"):
                traffic = float(line.split(":")[1]) * float(iters.size)

    def _accuracy_section():
        # per-result error against the FP64 oracle on a sample of the measured
        # population: 8 candidates x 16 lambdas, the same problem arrays, at
        # the benchmark's tolerance and at the tighter internal tolerance
        from oracle.solve import Problem as OracleProblem, eval_candidate
        n_acc = 8
        idx = np.arange(0, N_CAND, N_CAND // n_acc)[:n_acc]
        g = wl.geom
        f64 = lambda t: t.double().cpu().numpy().reshape(g.ny, g.nx)
        oprob = OracleProblem(g, f64(wl.problem.d), f64(wl.problem.sigma),
                              wl.problem.mask.cpu().numpy().reshape(g.ny, g.nx),
                              wl.problem.psf.double().cpu().numpy().reshape(g.kpsf, g.kpsf))
        lams = wl.lambdas[0].cpu().numpy()
        lens_h = wl.lens.cpu().numpy()
        t0 = time.perf_counter()
        refs = [eval_candidate(oprob, lens_h[c], lams) for c in idx]
        t_oracle = time.perf_counter() - t0
        sel = torch.as_tensor(idx, device="cuda")
        acc = {"sample": f"{n_acc} candidates x {N_LAM} lambdas of the timed population (FP64 dense-Cholesky oracle)",
               "oracle_s": t_oracle}
        for name, tol in (("tol_1e-6", TOL), (f"tol_{TIGHT_TOL:g}", TIGHT_TOL)):
            sub = ctx.eval_batch(probs, wl.lens[sel].contiguous(), wl.prob_idx[idx], wl.lambdas[sel].contiguous(),
                                 wl.n_lam[idx], tol=tol, maxit=100000, want_all_x=True)
            X = sub["all_x"].double().cpu().numpy()
            chi = sub["chi2"].cpu().numpy()
            ist = sub["item_status"].cpu().numpy()
            ce, se = [], []
            for j, r in enumerate(refs):
                ce += list(np.abs(chi[j] - r.chi2) / r.chi2)
                se += [np.linalg.norm(X[j, k, :g.ns] - r.s[k]) / np.linalg.norm(r.s[k]) for k in range(N_LAM)]
            ce, se = np.array(ce), np.array(se)
            acc[name] = {"chi2_rel_err_max": float(ce.max()), "chi2_rel_err_median": float(np.median(ce)),
                         "items_chi2_over_1e-5": int((ce > 1e-5).sum()),
                         "s_rel_err_max": float(se.max()), "s_rel_err_median": float(np.median(se)),
                         "items_s_over_1e-4": int((se > 1e-4).sum()), "items": int(ce.size),
                         "items_flagged": int(((ist & 7) != 0).sum())}
            if tol == TOL:
                # the sampled candidates' results are those of the timed step
                acc[name]["identical_to_timed_step"] = bool(np.array_equal(chi, out["chi2"][sel].cpu().numpy()))
        return acc

    acc_res = _guarded("accuracy", _accuracy_section)

    def _tight_section():
        # the whole population at the tighter internal tolerance, where every
        # sampled result meets |ds|/|s| <= 1e-4 and |dchi2|/chi2 <= 1e-5
        tout = ctx.eval_batch(probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=TIGHT_TOL, maxit=100000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        tout = ctx.eval_batch(probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=TIGHT_TOL, maxit=100000,
                              out=tout)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return {"tol": TIGHT_TOL, "evals_per_s": N_CAND / (ms / 1e3), "ms": ms,
                "cg_iters_mean_per_item": float(tout["iters"].float().mean().item()),
                "items_flagged": int(((tout["item_status"] & 7) != 0).sum().item())}

    tight_res = _guarded("tight_tolerance", _tight_section)

    def _tf32_section():
        # the inner solves' convolutions at TF32 precision (variant 7: both
        # factors of every product rounded to 10-bit mantissas, FP32 sums):
        # what a single-pass TF32 tensor-core B/B^T would cost in CG
        # iterations inside the exact FP64 refinement
        res = {"note": "FFMA kernel with TF32-rounded factors (a precision experiment, not a tensor-core kernel)"}
        for name, var in (("fp32", variant), ("tf32_factors", 7)):
            o = ctx.eval_batch(probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=TOL, variant=var)
            o, ms = _timed_call(lambda: ctx.eval_batch(probs, wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam,
                                                       tol=TOL, variant=var))
            it = o["iters"].float()
            res[name] = {"ms": ms, "cg_iters_mean_per_item": float(it.mean().item()),
                         "cg_iters_max": int(it.max().item()),
                         "items_flagged": int(((o["item_status"] & 7) != 0).sum().item()),
                         "relres_max": float(o["relres"].max().item())}
        res["iteration_ratio"] = res["tf32_factors"]["cg_iters_mean_per_item"] / res["fp32"]["cg_iters_mean_per_item"]
        return res

    tf32_res = _guarded("tf32_precision", _tf32_section)
    tcblur_res = _guarded("tc_blur", blur_engine_compare) if rank == 0 else None

    def _iter_section():
        # the paper's own fitness: 40 CGLS iterations per candidate, L-curve over
        # the iterations, Monte Carlo degrees of freedom (FP64 arithmetic)
        bh = torch.as_tensor(np.random.default_rng(5).standard_normal((1, wl.geom.nx * wl.geom.ny)),
                             dtype=ctx.real, device="cuda")
        iter_res = {"n_iter": 40}
        for key, b in (("evals_per_s", None), ("evals_per_s_with_dof", bh)):
            ctx.eval_iter(probs, wl.lens, wl.prob_idx, 40, bhat=b)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            io = ctx.eval_iter(probs, wl.lens, wl.prob_idx, 40, bhat=b)
            e1.record()
            torch.cuda.synchronize()
            iter_res[key] = N_CAND / (e0.elapsed_time(e1) / 1e3)
        cn = io["corner"].cpu().numpy()
        chi_c = io["chi2"].cpu().numpy()[np.arange(N_CAND), cn]
        dof_c = io["dof"].cpu().numpy()[np.arange(N_CAND), cn]
        iter_res.update({"corner_iteration_median": float(np.median(cn)),
                         "reduced_chi2_at_corner_median": float(np.median(chi_c / dof_c))})
        return iter_res

    iter_res = _guarded("iter_lcurve", _iter_section)

    def _forward_section():
        # forward batch (B L s and chi^2 of 1024 sources at one lens): 256x256
        # image at 0.02"/px, 128x128 source over +-1.2", 21x21 PSF; sources
        # |N(0,1)| times an analytic template
        import synth
        from paper_1101_5803_gb300.problems import large_workload
        lw = large_workload(ctx, n_cand=1, n_lam=1, seed=3)
        lg = lw.geom
        hx = (lg.sxmax - lg.sxmin) / lg.sx
        cxs = lg.sxmin + (np.arange(lg.sx) + 0.5) * hx
        tmpl = synth.eval_source(synth.drawn_source(np.random.default_rng(9)), *np.meshgrid(cxs, cxs)).ravel()
        n_src = 1024
        S = torch.as_tensor(np.abs(np.random.default_rng(10).standard_normal((n_src, tmpl.size))) * tmpl[None, :],
                            dtype=ctx.real, device="cuda")
        ctx.forward(lw.problem, lw.lens[0], S, want_model=False)  # warm-up
        fms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.forward(lw.problem, lw.lens[0], S, want_model=False)
            e1.record()
            torch.cuda.synchronize()
            fms.append(e0.elapsed_time(e1))
        npx = lg.nx * lg.ny
        fwd_flops = n_src * (2.0 * lg.kpsf * lg.kpsf * npx + 11.0 * npx)
        fwd_res = {"workload": "256x256 image, 128x128 source, 21x21 PSF, 1024 sources at one lens",
                   "ms": min(fms), "sources_per_s": n_src / (min(fms) / 1e3),
                   "tflops": fwd_flops / (min(fms) / 1e3) / 1e12}
        del S
        return fwd_res

    fwd_res = _guarded("forward_batch", _forward_section)

    def _wide_section():
        # a 65 x 65 PSF on the 64x64 system: the FFT blur (the automatic choice
        # at this width) against direct convolution (variant 6)
        from paper_1101_5803_gb300.problems import widepsf_workload
        ww = widepsf_workload(ctx, 16, 8, seed=5)
        wide = {"workload": "64x64 image, 32x32 source, 65x65 PSF, 16 candidates x 8 lambdas (1e-3..1e1)"}
        for name, var in (("fft", 0), ("direct", 6)):
            ctx.eval_batch([ww.problem], ww.lens[:2], ww.prob_idx[:2], ww.lambdas[:2], ww.n_lam[:2], tol=1e-6,
                           variant=var)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            wout = ctx.eval_batch([ww.problem], ww.lens, ww.prob_idx, ww.lambdas, ww.n_lam, tol=1e-6, variant=var)
            e1.record()
            torch.cuda.synchronize()
            wms = e0.elapsed_time(e1)
            wit = wout["iters"].cpu().numpy()
            wide[name] = {"ms": wms, "evals_per_s": 16 / (wms / 1e3), "cg_iterations": int(wit.sum()),
                          "us_per_iteration_of_slowest_item": wms * 1e3 / max(1, int(wit.max())),
                          "status_bits_any": int(np.bitwise_or.reduce(wout["status"].cpu().numpy()))}
        return wide

    wide = _guarded("wide_psf", _wide_section)

    n_gen = int(os.environ.get("MIRAGE_GA_GENERATIONS", "8"))

    def _ga_section():
        # GA generations on the same problem: the surrogate screen (4x
        # oversampled offspring, network trained beside the solves, lambda
        # chains from its predicted corner) against no screen
        from paper_1101_5803_gb300.ga import GAConfig, run_ga
        ga_res = {}
        for name, sur_on in (("with_surrogate", True), ("without", False)):
            cfg = GAConfig(pop=N_CAND, generations=n_gen, surrogate=sur_on, lam_chain=sur_on, seed=7)
            hist, _, bchi = run_ga(ctx, wl, cfg)
            gens = hist[1:]
            t_gen = sum(h.seconds for h in gens)
            ex = sum(h.exact_evals for h in gens)
            ga_res[name] = {"exact_evals_per_s": ex / t_gen,
                            "decisions_per_s": sum(h.decisions for h in gens) / t_gen,
                            "cg_iters_per_exact_eval": sum(h.cg_iters for h in gens) / max(1, ex),
                            "best_chi2_by_gen": [round(h.best_chi2, 2) for h in hist],
                            "seconds_by_gen": [round(h.seconds, 4) for h in hist],
                            "screened_gens": int(sum(h.screened for h in gens)),
                            "rank_corr_by_gen": [None if h.surrogate_rho is None else round(h.surrogate_rho, 3)
                                                 for h in gens],
                            "surrogate_rmse_by_gen": [None if h.surrogate_rmse is None else round(h.surrogate_rmse, 4)
                                                      for h in gens],
                            "fallback_rate": (1.0 - sum(h.screened for h in gens) / max(1, len(gens))) if sur_on else None}
        # best chi^2 of each run at the wall time at which the faster run ended
        # (generation 0, the shared initial population, excluded from the clock)
        def best_at(r, t):
            cum = np.cumsum(r["seconds_by_gen"][1:])
            k = int(np.searchsorted(cum, t * (1 + 1e-9), side="right"))
            return r["best_chi2_by_gen"][k]
        t_eq = min(sum(ga_res[k]["seconds_by_gen"][1:]) for k in ("with_surrogate", "without"))
        ga_res["best_chi2_at_equal_time"] = {"seconds": round(t_eq, 3),
                                             **{k: best_at(ga_res[k], t_eq) for k in ("with_surrogate", "without")}}
        ga_res["generations"] = n_gen
        ga_res["oversample"] = 4
        ga_res["note"] = ("decisions = offspring ranked per second (surrogate screen, then the exact solve of the "
                          "pop best); every survivor's fitness comes from the exact solve")
        return ga_res

    ga_res = _guarded("ga_surrogate", _ga_section)

    def _pso_section():
        # particle swarm (Eq. PSO) on the same problem: one batched call per step
        from paper_1101_5803_gb300.pso import PSOConfig, batch_evaluator, run_pso
        phist, _, _ = run_pso(batch_evaluator(ctx, wl), PSOConfig(particles=N_CAND, steps=n_gen, seed=7))
        psteps = phist[1:]
        t_pso = sum(h.seconds for h in psteps)
        pso_res = {"particles": N_CAND, "steps": n_gen,
                   "exact_evals_per_s": sum(h.evals for h in psteps) / t_pso,
                   "cg_iters_per_exact_eval": sum(h.cg_iters for h in psteps) / max(1, sum(h.evals for h in psteps)),
                   "best_chi2_by_step": [round(h.best_chi2, 2) for h in phist]}
        return pso_res

    pso_res = _guarded("pso", _pso_section)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, done, dt = oracle_evals_per_s(64, seed=7, budget_s=float(os.environ.get("MIRAGE_CPU_BUDGET", "20")))
        cpu = {"value": v, "unit": UNIT, "cores": _cpu_threads(), "kind": "oracle",
               "sample": f"{done} candidates x {N_LAM} lambdas of the same workload in {dt:.1f} s "
                         f"(dense Cholesky FP64)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 reductions)", "data": "synthetic",
            "config": dict(CONFIG, parallelism=f"replicas{world}" if world > 1 else "single",
                           kernel_variant=variant, tuned=tcfg),
            "e2e": {"value": N_CAND / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_basis": f"FP32 FFMA: {nsm} SMs x 128 lanes x 2 x {smax:.0f} MHz ({src} max clock)",
                         "frac_at_measured_clock": (achieved / at_clock) if at_clock else None,
                         "kernel": kernel_name, "kernel_ms": phase[1], "flops_per_launch": flops,
                         "ffma_microbench": {"tflops": ffma_tf, "flop_per_clk_per_sm_at_max_clock": ffma_fc,
                                             "frac_of_nominal": ffma_fc / 256.0,
                                             "kernel_frac_of_measured": achieved / ffma_tf}},
            "cpu_baseline": cpu,
            "plain": {"value": plain, "unit": UNIT, "sample": n_plain, "speedup_batched_vs_plain": value / plain,
                      "chi2_identical": same},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
            "cg": {"iters_mean_per_item": float(iters.mean()), "iters_max": int(iters.max()),
                   "relres_true_max": float(relres.max()), "relres_true_median": float(np.median(relres)),
                   "items_converged_frac": float(((item_status & 7) == 0).mean()),
                   "status_bits_any": int(np.bitwise_or.reduce(status))},
            "phase_ms": {"raytrace": phase[0], "cgls": phase[1], "finalize": phase[2]},
            "batched_surrogate": (None if "with_surrogate" not in ga_res else {
                "decisions_per_s": ga_res["with_surrogate"]["decisions_per_s"],
                "exact_evals_per_s": ga_res["with_surrogate"]["exact_evals_per_s"],
                "speedup_vs_plain": ga_res["with_surrogate"]["decisions_per_s"] / plain,
                "exact_speedup_vs_plain": ga_res["with_surrogate"]["exact_evals_per_s"] / plain,
                "exact_evals_per_s_without_surrogate": ga_res["without"]["exact_evals_per_s"],
                "workload": f"GA on the same problem, population {N_CAND}, {n_gen} generations, 4x oversampled "
                            f"offspring"}),
            "accuracy": acc_res,
            "tight_tolerance": tight_res,
            "tf32_precision": tf32_res,
            "tc_blur": tcblur_res,
            "ga_surrogate": ga_res,
            "pso": pso_res,
            "iter_lcurve": iter_res,
            "forward_batch": fwd_res,
            "wide_psf": wide}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile_case(variant: int, n_cand: int = 160) -> int:
    """The case the ncu captures of the CGLS kernel run: n_cand candidates x
    the 16-lambda grid of the 64x64 workload (160 x 16 = 2560 items, over
    eight per CTA slot of the two-CTA kernel, so the launch is in the
    benchmark's steady state), two evaluations with one kernel variant, then
    one with per-phase SM clocks; no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import ga64_workload
    ctx = binding.Context(0, binding.MIRAGE_FP32)
    wl = ga64_workload(ctx, n_cand, 16, seed=3)
    for _ in range(2):
        out = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, variant=variant)
    torch.cuda.synchronize()
    # one more evaluation with the two-CTA kernel's per-phase SM clocks
    ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, wl.lambdas, wl.n_lam, tol=1e-6, variant=variant,
                   phase_clocks=True)
    torch.cuda.synchronize()
    clk = [float(v) for v in ctx.phase_clocks()]
    its = float(out["iters"].sum().item())
    names = ["L p + H p", "B convolution + W q + H^T H p", "delta reduction", "(unused)", "B^T convolution", "L^T walk",
             "L^T join", "L^T gather + updates", "gamma reduction", "p update", "FP64 refinement", "item set-up"]
    print(json.dumps({"profile_case": True, "variant": variant, "items": int(out["iters"].numel()),
                      "cg_iterations": int(its),
                      "phase_clk_per_iteration": {n: round(c / max(its, 1.0), 1) for n, c in zip(names, clk)}}),
          flush=True)
    ctx.close()
    return 0


def blur_engine_compare(n: int = 4096, reps: int = 64, repeats: int = 3) -> dict:
    """The blur B of the inner solves (64 x 64 images, the workload's 9 x 9
    Gaussian PSF) on the CG kernel's FFMA register tiles and as TF32
    block-Toeplitz products on the tcgen05 tensor cores (mirage_psf_blur):
    n images, B applied `reps` times to each while it stays in shared
    memory, the fastest of `repeats` timed calls after a warm-up call."""
    import torch

    import synth
    from paper_1101_5803_gb300 import binding
    g = synth.geom_ga64()
    K = g.kpsf
    psf = synth.gaussian_psf(K, synth.PSF_SIGMA["ga64"]).astype(np.float32)
    imgs = torch.as_tensor(np.random.default_rng(11).standard_normal((n, g.ny, g.nx)).astype(np.float32),
                           device="cuda")
    out = torch.empty_like(imgs)
    flop = 2.0 * K * K * g.nx * g.ny
    # the products the tensor cores execute: 16-column strips, 128-row tiles
    # of the stacked strips, a 24-wide Toeplitz window per PSF row
    tiles = -(-(g.nx // 16) * (g.ny + K - 1) // 128)
    tc_flop = 2.0 * tiles * 128 * 16 * ((16 + K - 1 + 7) // 8 * 8) * K
    peaks, basis = measured_peaks()
    tf32_peak = peaks["bf16_tflops"] / 2.0
    res = {"images": n, "reps": reps, "image": [g.ny, g.nx], "kpsf": K, "algorithmic_flop_per_blur": flop,
           "tensor_flop_per_blur": tc_flop,
           "tf32_peak_tflops": tf32_peak, "tf32_peak_basis": f"{basis} bf16 x 1/2 (nominal TF32/BF16 ratio)"}
    one = {}
    for name, eng in (("ffma", binding.MIRAGE_BLUR_FFMA), ("tc_tf32", binding.MIRAGE_BLUR_TC_TF32)):
        binding.mirage_psf_blur(eng, imgs, psf, reps, out=out)
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            binding.mirage_psf_blur(eng, imgs, psf, reps, out=out)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        nb = n * reps
        r = {"ms": best, "ns_per_blur": best * 1e6 / nb, "tflops_algorithmic": flop * nb / (best * 1e-3) / 1e12}
        if eng == binding.MIRAGE_BLUR_TC_TF32:
            r["tflops_tensor"] = tc_flop * nb / (best * 1e-3) / 1e12
            r["frac_of_tf32_peak"] = r["tflops_tensor"] / tf32_peak
        res[name] = r
        one[name] = binding.mirage_psf_blur(eng, imgs[:256], psf, 1).double()
    res["tc_max_rel_diff_one_blur"] = float(((one["tc_tf32"] - one["ffma"]).abs().max() /
                                             one["ffma"].abs().max()).item())
    res["speedup_tc_over_ffma"] = res["ffma"]["ms"] / res["tc_tf32"]["ms"]
    return res


def run_blur_engines(n: int, reps: int) -> int:
    """The blur-engine comparison alone (also the case of its ncu captures)."""
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps({"blur_engines": blur_engine_compare(n, reps)}), flush=True)
    return 0


def run_profile_forward() -> int:
    """The case the ncu captures of the forward-batch kernel run: the
    256x256 forward batch of the benchmark (128x128 source, 21x21 PSF, 1024
    sources |N(0,1)| x template at one lens), three calls, no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import large_workload
    ctx = binding.Context(0, binding.MIRAGE_FP32)
    lw = large_workload(ctx, n_cand=1, n_lam=1, seed=3)
    lg = lw.geom
    hx = (lg.sxmax - lg.sxmin) / lg.sx
    cxs = lg.sxmin + (np.arange(lg.sx) + 0.5) * hx
    tmpl = synth.eval_source(synth.drawn_source(np.random.default_rng(9)), *np.meshgrid(cxs, cxs)).ravel()
    S = torch.as_tensor(np.abs(np.random.default_rng(10).standard_normal((1024, tmpl.size))) * tmpl[None, :],
                        dtype=ctx.real, device="cuda")
    for _ in range(3):
        _, chi2, _ = ctx.forward(lw.problem, lw.lens[0], S, want_model=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_forward": True, "sources": 1024, "chi2_median": float(chi2.median().item())}),
          flush=True)
    ctx.close()
    return 0


def _oracle_problem(prob, geom):
    """The oracle's view of a device problem: the same arrays in float64."""
    from oracle.solve import Problem as OracleProblem
    f64 = lambda t: t.double().cpu().numpy().reshape(geom.ny, geom.nx)
    return OracleProblem(geom, f64(prob.d), f64(prob.sigma), prob.mask.cpu().numpy().reshape(geom.ny, geom.nx),
                         prob.psf.double().cpu().numpy().reshape(geom.kpsf, geom.kpsf))


def _errs(chi, X, ns, ref, n):
    """Per-lambda |dchi2|/chi2 and |ds|/|s| of one candidate against an oracle result."""
    ce = np.abs(chi[:n] - ref.chi2[:n]) / ref.chi2[:n]
    se = np.array([np.linalg.norm(X[k, :ns] - ref.s[k]) / np.linalg.norm(ref.s[k]) for k in range(n)])
    return ce, se


def _summ(ce, se):
    ce, se = np.concatenate(ce), np.concatenate(se)
    return {"items": int(ce.size), "chi2_rel_err_max": float(ce.max()), "chi2_rel_err_median": float(np.median(ce)),
            "items_chi2_over_1e-5": int((ce > 1e-5).sum()), "s_rel_err_max": float(se.max()),
            "s_rel_err_median": float(np.median(se)), "items_s_over_1e-4": int((se > 1e-4).sum())}


def _timed_call(fn):
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    out = fn()
    e1.record(st)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def run_workload(name: str, args) -> int:
    """One of the other stated workloads at full size, with a sampled oracle
    check; prints one JSON line (not the default benchmark line)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from oracle.solve import eval_candidate
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300 import problems as P

    ctx = binding.Context(0, binding.MIRAGE_FP32)
    res = {"workload": name}
    if name == "uneven1024":
        # 1024 candidates, each with its own observation: images {48..128}^2 with
        # annular masks, sources {16..48}^2, PSFs {7,11,15}, 8..32 lambdas
        from paper_1101_5803_gb300.autotune import tune_config
        mw = P.uneven_workload(ctx, 1024, seed=1)
        call = lambda **kw: ctx.eval_batch(mw.problems, mw.lens, mw.prob_idx, mw.lambdas, mw.n_lam, tol=TOL, **kw)
        call()  # warm-up (kernel attributes, scratch)
        _, ms_default = _timed_call(call)
        # the autotuner's configuration for this shape class (probe: the first
        # 64 candidates' grids), then the timed full batch with it
        tcfg = tune_config(ctx, mw.problems, mw.lens, mw.prob_idx, mw.lambdas, mw.n_lam, tol=TOL)
        call(**tcfg)
        _, ms = _timed_call(lambda: call(**tcfg))
        out = call(want_all_x=True, **tcfg)  # the same results, with every lambda's source for the oracle check
        res["autotune"] = {"config": tcfg, "ms_default": ms_default, "ms_tuned": ms,
                           "gain": ms_default / ms}
        ist = out["item_status"].cpu().numpy()
        valid = np.arange(ist.shape[1])[None, :] < mw.n_lam[:, None]
        res.update({"config": "1024 candidates, images {48,64,96,128}^2 (6.4\"), annular masks 0.3-0.6\" / "
                              "1.5-2.5\", sources {16,24,32,48}^2 over +-0.8\", PSFs {7,11,15} px, 8-32 lambdas "
                              "1e-4..1e2, tol 1e-6, one call",
                    "ms": ms, "evals_per_s": 1024 / (ms / 1e3), "items": int(valid.sum()),
                    "cg_iterations": int(out["iters"].cpu().numpy()[valid].sum()),
                    "items_converged_frac": float(((ist & 7) == 0)[valid].mean()),
                    "status_bits_any": int(np.bitwise_or.reduce(out["status"].cpu().numpy()))})
        # oracle on 16 sampled candidates (every image size, their own lambda grids)
        rng = np.random.default_rng(3)
        pick = np.sort(rng.choice(1024, 16, replace=False))
        X = out["all_x"].double().cpu().numpy()
        chi = out["chi2"].cpu().numpy()
        lens_h = mw.lens.cpu().numpy()
        lam_h = mw.lambdas.cpu().numpy()
        ce, se = [], []
        t0 = time.perf_counter()
        refs = {}
        for c in pick:
            pr = mw.problems[c]
            r = refs[c] = eval_candidate(_oracle_problem(pr, pr.geom), lens_h[c], lam_h[c, :mw.n_lam[c]])
            a, b = _errs(chi[c], X[c], pr.geom.ns, r, mw.n_lam[c])
            ce.append(a)
            se.append(b)
        res["oracle_sample"] = dict(_summ(ce, se), candidates=[int(c) for c in pick],
                                    oracle_s=time.perf_counter() - t0)
        # the same candidates at the tighter internal tolerance
        sel = torch.as_tensor(pick, device="cuda")
        tout = ctx.eval_batch([mw.problems[c] for c in pick], mw.lens[sel].contiguous(),
                              np.arange(len(pick), dtype=np.int32), mw.lambdas[sel].contiguous(), mw.n_lam[pick],
                              tol=TIGHT_TOL, maxit=200000, want_all_x=True)
        Xt = tout["all_x"].double().cpu().numpy()
        ct = tout["chi2"].cpu().numpy()
        ce, se = [], []
        for j, c in enumerate(pick):
            a, b = _errs(ct[j], Xt[j], mw.problems[c].geom.ns, refs[c], mw.n_lam[c])
            ce.append(a)
            se.append(b)
        res[f"oracle_sample_tol_{TIGHT_TOL:g}"] = dict(_summ(ce, se), items_flagged=int(
            ((tout["item_status"].cpu().numpy() & 7) != 0)[np.arange(tout["item_status"].shape[1])[None, :]
                                                             < mw.n_lam[pick][:, None]].sum()))
    elif name == "ga128":
        # the end-to-end GA: 128x128 image at 0.03", 48x48 source, 11x11 PSF,
        # population 512 x G generations, 4x oversampled surrogate screen
        from paper_1101_5803_gb300.ga import GAConfig, run_ga
        gens = args.generations
        wl = P.e2e128_workload(ctx, n_cand=512, seed=0)
        cfg = GAConfig(pop=512, generations=gens, surrogate=True, lam_chain=True, seed=0)
        hist, best, bchi = run_ga(ctx, wl, cfg)
        g = hist[1:]
        tg = sum(h.seconds for h in g)
        rms = [h.surrogate_rmse for h in g if h.surrogate_rmse is not None]
        res.update({"config": f"128x128 image 0.03\"/px, 48x48 source +-0.8\", 11x11 PSF sigma 1.5 px, Laplacian, "
                              f"16 lambdas 1e-4..1e2, population 512 x {gens} generations, 4x oversampled screen",
                    "seconds": tg, "exact_evals_per_s": sum(h.exact_evals for h in g) / tg,
                    "decisions_per_s": sum(h.decisions for h in g) / tg,
                    "fallback_rate": 1.0 - sum(h.screened for h in g) / max(1, len(g)),
                    "surrogate_rmse_first_last_median": [rms[0], rms[-1], float(np.median(rms))] if rms else None,
                    "surrogate_rmse_by_gen": [None if h.surrogate_rmse is None else round(h.surrogate_rmse, 4) for h in g],
                    "rank_corr_by_gen": [None if h.surrogate_rho is None else round(h.surrogate_rho, 3) for h in g],
                    "best_chi2_by_gen": [round(h.best_chi2, 2) for h in hist],
                    "best_lens": [float(v) for v in best], "best_chi2": bchi,
                    "true_lens": [float(v) for v in __import__("synth").TRUE_LENS]})
        # oracle on the best lens: the exact solve's corner chi^2 and every lambda
        lams = wl.lambdas[0].cpu().numpy()
        out = ctx.eval_batch([wl.problem], torch.as_tensor(best[None, :], device="cuda"), [0], wl.lambdas[:1],
                             wl.n_lam[:1], tol=TOL, want_all_x=True)
        t0 = time.perf_counter()
        r = eval_candidate(_oracle_problem(wl.problem, wl.geom), best, lams)
        a, b = _errs(out["chi2"][0].cpu().numpy(), out["all_x"][0].double().cpu().numpy(), wl.geom.ns, r, len(lams))
        res["oracle_best_lens"] = dict(_summ([a], [b]), corner_gpu=int(out["corner"][0].item()), corner_oracle=r.corner,
                                       oracle_s=time.perf_counter() - t0)
    elif name == "large256":
        # 64 candidates x 32 lambdas at 256x256 (128x128 source, 21x21 PSF),
        # CG to 1e-6, with and without the surrogate's predicted lambda*
        # starting each candidate's chains
        from oracle.cg import chi2_reg, cgls_solve, sparse_operators
        from paper_1101_5803_gb300.ga import Surrogate
        n_c, n_l = 64, 32
        wl = P.large_workload(ctx, n_cand=n_c + 16, n_lam=n_l, seed=3)
        lams = wl.lambdas[0].cpu().numpy()
        # the surrogate learns (log chi2*, log10 lambda*) from 16 other candidates
        tr = slice(n_c, n_c + 16)
        tout = ctx.eval_batch([wl.problem], wl.lens[tr].contiguous(), wl.prob_idx[tr], wl.lambdas[tr].contiguous(),
                              wl.n_lam[tr], tol=TOL)
        tc = tout["corner"].cpu().numpy()
        tchi = tout["chi2"].cpu().numpy()[np.arange(16), tc]
        sur = Surrogate(256, 0)
        sur.add(wl.lens[tr].cpu().numpy(), tchi, lams[tc])
        sur.train(600, 16, 2e-3, np.random.default_rng(0))
        lens_m = wl.lens[:n_c].contiguous()
        l10 = sur.predict(lens_m.cpu().numpy())[:, 1] * sur.ysd[1] + sur.ymu[1]
        ks = np.abs(np.log10(lams)[None, :] - l10[:, None]).argmin(axis=1).astype(np.int32)
        runs = {}
        for key, kw in (("cold", {}), ("surrogate_lambda_start", {"lam_start": ks})):
            o, ms = _timed_call(lambda: ctx.eval_batch([wl.problem], lens_m, wl.prob_idx[:n_c],
                                                       wl.lambdas[:n_c].contiguous(), wl.n_lam[:n_c], tol=TOL,
                                                       want_all_x=(key == "cold"), **kw))
            it = o["iters"].cpu().numpy()
            runs[key] = {"ms": ms, "evals_per_s": n_c / (ms / 1e3), "cg_iterations": int(it.sum()),
                         "cg_iterations_max_item": int(it.max()),
                         "items_converged_frac": float(((o["item_status"].cpu().numpy() & 7) == 0).mean()),
                         "out": o}
        cold = runs["cold"].pop("out")
        warm = runs["surrogate_lambda_start"].pop("out")
        npix = wl.geom.nx * wl.geom.ny
        f_it = 4 * 21 * 21 * npix + 16 * npix + 32 * wl.geom.ns
        for key in runs:
            runs[key]["tflops"] = runs[key]["cg_iterations"] * f_it / (runs[key]["ms"] / 1e3) / 1e12
        res.update({"config": "256x256 image 0.02\"/px, 128x128 source +-1.2\", 21x21 PSF sigma 3 px, Laplacian, "
                              "64 candidates x 32 lambdas 1e-4..1e2, tol 1e-6",
                    "runs": runs,
                    "chi2_agree_cold_vs_warm_max_rel": float(np.max(np.abs(warm["chi2"].cpu().numpy() -
                                                                          cold["chi2"].cpu().numpy()) /
                                                                   cold["chi2"].cpu().numpy()))})
        # matrix-free FP64 oracle (dense F does not fit) on 2 candidates x the 2
        # largest lambdas (the oracle's CGLS needs far fewer iterations there)
        op = _oracle_problem(wl.problem, wl.geom)
        X = cold["all_x"].double().cpu().numpy()
        chi = cold["chi2"].cpu().numpy()
        ce, se = [], []
        t0 = time.perf_counter()
        for c in (0, 1):
            ops = sparse_operators(op, wl.lens[c].cpu().numpy())
            for k in (n_l - 2, n_l - 1):
                s_ref, _, _ = cgls_solve(ops, float(lams[k]), tol=1e-12)
                c_ref, _ = chi2_reg(ops, s_ref)
                ce.append(np.array([abs(chi[c, k] - c_ref) / c_ref]))
                se.append(np.array([np.linalg.norm(X[c, k, :wl.geom.ns] - s_ref) / np.linalg.norm(s_ref)]))
        res["oracle_sample"] = dict(_summ(ce, se), sample="candidates 0-1 x the two largest lambdas, matrix-free "
                                                          "FP64 CGLS oracle at tol 1e-12",
                                    oracle_s=time.perf_counter() - t0)
    else:
        raise SystemExit(f"unknown workload {name}")
    print(json.dumps(res), flush=True)
    ctx.close()
    return 0


def run_profile_large() -> int:
    """The case the ncu captures of the general CGLS kernel at 256x256 run
    (all work vectors in the CTA's global slab, two CTAs per SM): 304
    candidates x lambda = 10 (one item per CTA slot), two evaluations."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    from paper_1101_5803_gb300.problems import large_workload
    ctx = binding.Context(0, binding.MIRAGE_FP32)
    n = 304
    wl = large_workload(ctx, n_cand=n, n_lam=1, seed=3)
    lam = torch.full((n, 1), 10.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out = ctx.eval_batch([wl.problem], wl.lens, wl.prob_idx, lam, wl.n_lam, tol=TOL)
    torch.cuda.synchronize()
    print(json.dumps({"profile_large": True, "items": n, "cg_iterations": int(out["iters"].sum().item()),
                      "iters_max": int(out["iters"].max().item()),
                      "converged": bool(((out["item_status"] & 7) == 0).all().item())}), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-case", type=int, default=None, metavar="VARIANT",
                    help="run only the case of the ncu captures of the CGLS kernel (--profile-cands "
                         "candidates x 16 lambdas, two evaluations with this kernel variant) and exit")
    ap.add_argument("--profile-cands", type=int, default=160,
                    help="candidates of the --profile-case run (x 16 lambdas)")
    ap.add_argument("--profile-forward", action="store_true",
                    help="run only the forward-batch case of the ncu captures (256x256, 1024 sources) and exit")
    ap.add_argument("--profile-large", action="store_true",
                    help="run only the 256x256 case of the ncu captures of the general CGLS kernel and exit")
    ap.add_argument("--workload", default=None, choices=["uneven1024", "ga128", "large256"],
                    help="run one of the other stated workloads at full size with a sampled oracle check and "
                         "print its own JSON line")
    ap.add_argument("--generations", type=int, default=200, help="generations of --workload ga128")
    ap.add_argument("--blur-engines", action="store_true",
                    help="run only the blur-engine comparison (FFMA tiles against tcgen05 TF32) and exit")
    ap.add_argument("--blur-images", type=int, default=4096, help="images of --blur-engines")
    ap.add_argument("--blur-reps", type=int, default=64, help="applications of B per image in --blur-engines")
    args = ap.parse_args()
    if args.blur_engines:
        return run_blur_engines(args.blur_images, args.blur_reps)
    if args.workload:
        return run_workload(args.workload, args)
    if args.profile_large:
        return run_profile_large()
    if args.profile_forward:
        return run_profile_forward()
    if args.profile_case is not None:
        return run_profile_case(args.profile_case, args.profile_cands)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
