"""Thin ctypes binding of libmirage (include/mirage.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  Functions carry the C names; tensors are passed by pointer.
Device tensors go to the device path; CPU tensors (ideally pinned) go to the
``MIRAGE_MEM_HOST`` path, which stages them inside the library.

There is no CPU fallback: if the compiled library is missing, loading fails
with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmirage.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mirage.h")

MIRAGE_OK = 0
MIRAGE_FP32, MIRAGE_FP64 = 0, 1
MIRAGE_MEM_DEVICE, MIRAGE_MEM_HOST = 0, 1
MIRAGE_MODE_BATCHED, MIRAGE_MODE_PLAIN = 0, 1
MIRAGE_INTERP_BILINEAR, MIRAGE_INTERP_NEAREST, MIRAGE_INTERP_BICUBIC = 0, 1, 2
MIRAGE_REG_IDENTITY, MIRAGE_REG_GRADIENT, MIRAGE_REG_LAPLACIAN = 0, 1, 2
MIRAGE_BLUR_FFMA, MIRAGE_BLUR_TC_TF32 = 0, 1
ST_MAXIT, ST_STAGNATION, ST_BREAKDOWN, ST_BAD_PARAM, ST_EMPTY_MAP, ST_LCURVE_FLAT = 1, 2, 4, 8, 16, 32
MAX_LAM = 64
MAX_KPSF = 65  # MIRAGE_MAX_KPSF
N_PHASE_CLOCKS = 12  # MIRAGE_N_PHASE_CLOCKS


class MirageError(RuntimeError):
    pass


class mirage_geom_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pix", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("sx", ctypes.c_int),
                ("sy", ctypes.c_int), ("sxmin", ctypes.c_double), ("sxmax", ctypes.c_double),
                ("symin", ctypes.c_double), ("symax", ctypes.c_double), ("kpsf", ctypes.c_int),
                ("subpix", ctypes.c_int), ("reg", ctypes.c_int), ("interp", ctypes.c_int)]


class mirage_problem_t(ctypes.Structure):
    _fields_ = [("geom", mirage_geom_t), ("d", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("psf", ctypes.c_void_p)]


class mirage_opts_t(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("mode", ctypes.c_int),
                ("mem", ctypes.c_int), ("use_graph", ctypes.c_int), ("threads", ctypes.c_int),
                ("replace_every", ctypes.c_int), ("variant", ctypes.c_int), ("inner_eta", ctypes.c_double),
                ("place", ctypes.c_int)]


_lib = None


def load_library():
    """Load libmirage.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MirageError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                          f"g.build()\"` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double
    lib.mirage_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i, i]
    lib.mirage_create.restype = ip
    lib.mirage_destroy.argtypes = [vp]
    lib.mirage_destroy.restype = ip
    lib.mirage_eval_batch.argtypes = [vp, ctypes.POINTER(mirage_problem_t), i, vp, vp, i, vp, vp, i,
                                      ctypes.POINTER(mirage_opts_t), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      vp, vp, vp]
    lib.mirage_eval_batch.restype = ip
    lib.mirage_lcurve.argtypes = [vp, vp, vp, i, i, vp, vp, vp, vp]
    lib.mirage_lcurve.restype = ip
    lib.mirage_forward.argtypes = [vp, ctypes.POINTER(mirage_problem_t), vp, vp, i, vp, vp, vp, vp]
    lib.mirage_forward.restype = ip
    lib.mirage_eval_iter.argtypes = [vp, ctypes.POINTER(mirage_problem_t), i, vp, vp, i, i, vp, ctypes.c_longlong,
                                     vp, vp, vp, vp, vp, vp, vp, vp]
    lib.mirage_eval_iter.restype = ip
    lib.mirage_measure_ffma.argtypes = [i, vp, vp]
    lib.mirage_measure_ffma.restype = ip
    lib.mirage_set_reserved_slots.argtypes = [vp, i]
    lib.mirage_set_reserved_slots.restype = ip
    lib.mirage_last_launch_count.argtypes = [vp]
    lib.mirage_last_launch_count.restype = ip
    lib.mirage_last_phase_clocks.argtypes = [vp, vp]
    lib.mirage_last_phase_clocks.restype = ip
    lib.mirage_last_phase_ms.argtypes = [vp, vp]
    lib.mirage_last_phase_ms.restype = ip
    lib.mirage_last_error.argtypes = []
    lib.mirage_last_error.restype = ctypes.c_char_p
    lib.mirage_forward_noalloc.argtypes = [i, ctypes.POINTER(mirage_problem_t), vp, vp, i, vp, vp, vp, vp]
    lib.mirage_forward_noalloc.restype = ip
    lib.mirage_noalloc_last_error.argtypes = []
    lib.mirage_noalloc_last_error.restype = ctypes.c_char_p
    lib.mirage_psf_blur.argtypes = [i, vp, vp, i, i, i, vp, i, i, vp]
    lib.mirage_psf_blur.restype = ip
    lib.mirage_blur_last_error.argtypes = []
    lib.mirage_blur_last_error.restype = ctypes.c_char_p
    lib.mirage_noalloc_capacity.argtypes = []
    lib.mirage_noalloc_capacity.restype = ctypes.c_size_t
    ll = ctypes.c_long
    lib.mirage_mlp_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i, i, vp, ctypes.c_ulonglong]
    lib.mirage_mlp_create.restype = ip
    lib.mirage_mlp_destroy.argtypes = [vp]
    lib.mirage_mlp_destroy.restype = ip
    lib.mirage_mlp_num_params.argtypes = [vp]
    lib.mirage_mlp_num_params.restype = ll
    lib.mirage_mlp_set_params.argtypes = [vp, vp, ll]
    lib.mirage_mlp_set_params.restype = ip
    lib.mirage_mlp_get_params.argtypes = [vp, vp, ll]
    lib.mirage_mlp_get_params.restype = ip
    lib.mirage_mlp_forward.argtypes = [vp, vp, i, vp, vp]
    lib.mirage_mlp_forward.restype = ip
    lib.mirage_mlp_grad.argtypes = [vp, vp, vp, i, vp, vp, vp, vp]
    lib.mirage_mlp_grad.restype = ip
    lib.mirage_mlp_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, vp, vp, vp]
    lib.mirage_mlp_train_step.restype = ip
    lib.mirage_mlp_train.argtypes = [vp, vp, vp, i, i, i, ctypes.c_float, ctypes.c_ulonglong, vp]
    lib.mirage_mlp_train.restype = ip
    lib.mirage_mlp_last_error.argtypes = []
    lib.mirage_mlp_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions include/mirage.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long|size_t|const char\*)\s+(mirage_\w+)\s*\(", txt, re.M)))


def _check(rc: int, what: str):
    if rc != MIRAGE_OK:
        msg = load_library().mirage_last_error().decode(errors="replace")
        raise MirageError(f"{what} failed ({rc}): {msg}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Problem:
    """Geometry (any object with the mirage_geom_t field names) plus data tensors.

    ``d``, ``sigma``, ``psf`` are float32 (FP32 contexts) or float64 (FP64
    contexts) tensors, ``mask`` uint8; all on the device, or all on the host
    for the host-memory path.
    """

    def __init__(self, geom, d, sigma, mask, psf):
        self.geom = geom
        self.d, self.sigma, self.mask, self.psf = d.contiguous(), sigma.contiguous(), mask.contiguous(), psf.contiguous()

    def c_struct(self) -> mirage_problem_t:
        g = self.geom
        cg = mirage_geom_t(int(g.nx), int(g.ny), float(g.pix), float(getattr(g, "cx", 0.0)),
                           float(getattr(g, "cy", 0.0)), int(g.sx), int(g.sy), float(g.sxmin), float(g.sxmax),
                           float(g.symin), float(g.symax), int(g.kpsf), int(getattr(g, "subpix", 1)), int(g.reg),
                           int(getattr(g, "interp", 0)))
        return mirage_problem_t(cg, self.d.data_ptr(), self.sigma.data_ptr(), self.mask.data_ptr(),
                                self.psf.data_ptr())


def mirage_create(device: int = 0, precision: int = MIRAGE_FP32) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.mirage_create(ctypes.byref(h), device, precision), "mirage_create")
    return h


def mirage_destroy(ctx) -> None:
    _check(load_library().mirage_destroy(ctx), "mirage_destroy")


def mirage_last_launch_count(ctx) -> int:
    return int(load_library().mirage_last_launch_count(ctx))


def mirage_eval_batch(ctx, probs, lens, prob_idx, lambdas, n_lam, *, tol=1e-6, maxit=0,
                      mode=MIRAGE_MODE_BATCHED, use_graph=False, replace_every=0, warm_x=None, lam_start=None,
                      want_s=True, want_all_x=False, want_kappa=True, out=None, stream=None, real=torch.float32,
                      phase_timing=False, phase_clocks=False, variant=0, inner_eta=0.0, place=0):
    """Evaluate candidates; returns a dict of output tensors (see mirage.h).

    ``lens`` [n,7] float64 and ``lambdas`` [n,max_lam] float64 are device
    tensors (host tensors select the host-memory path); ``prob_idx`` and
    ``n_lam`` are host integer sequences.  ``out`` may pass preallocated
    outputs (same keys as the returned dict) to keep pointers stable for
    graph replay.  ``lam_start`` (host ints, one per candidate) solves each
    candidate's lambdas as warm-started chains from that index (mirage.h).
    """
    lib = load_library()
    n = int(lens.shape[0])
    max_lam = int(lambdas.shape[1])
    host = not lens.is_cuda
    dev = lens.device
    max_ns = max(int(p.geom.sx) * int(p.geom.sy) for p in probs)
    pidx = np.ascontiguousarray(np.asarray(prob_idx, dtype=np.int32))
    nl = np.ascontiguousarray(np.asarray(n_lam, dtype=np.int32))
    ls = None if lam_start is None else np.ascontiguousarray(np.asarray(lam_start, dtype=np.int32))
    if ls is not None and ls.shape != (n,):
        raise ValueError("lam_start needs one index per candidate")
    if out is None:
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, device=dev, pin_memory=host and torch.cuda.is_available())
        out = {"chi2": mk((n, max_lam), torch.float64), "reg": mk((n, max_lam), torch.float64),
               "iters": mk((n, max_lam), torch.int32), "relres": mk((n, max_lam), torch.float64),
               "item_status": mk((n, max_lam), torch.int32), "corner": mk((n,), torch.int32),
               "status": mk((n,), torch.int32)}
        if want_kappa:
            out["kappa"] = mk((n, max_lam), torch.float64)
        if want_s:
            out["s"] = mk((n, max_ns), real)
        if want_all_x:
            out["all_x"] = mk((n, max_lam, max_ns), real)
    arr = (mirage_problem_t * len(probs))(*[p.c_struct() for p in probs])
    opts = mirage_opts_t(float(tol), int(maxit), int(mode), MIRAGE_MEM_HOST if host else MIRAGE_MEM_DEVICE,
                         int(bool(use_graph)), -2 if phase_clocks else (-1 if phase_timing else 0),
                         int(replace_every), int(variant), float(inner_eta), int(place))
    rc = lib.mirage_eval_batch(
        ctx, arr, len(probs), _ptr(lens.contiguous()), pidx.ctypes.data_as(ctypes.c_void_p), n,
        _ptr(lambdas.contiguous()), nl.ctypes.data_as(ctypes.c_void_p), max_lam, ctypes.byref(opts),
        _ptr(warm_x), None if ls is None else ls.ctypes.data_as(ctypes.c_void_p), _ptr(out["chi2"]), _ptr(out["reg"]), _ptr(out["iters"]), _ptr(out.get("relres")),
        _ptr(out.get("item_status")), _ptr(out["corner"]), _ptr(out.get("kappa")), _ptr(out.get("s")),
        _ptr(out.get("all_x")), _ptr(out["status"]), None if host else _stream_ptr(stream))
    _check(rc, "mirage_eval_batch")
    return out


def mirage_last_phase_ms(ctx):
    """[ray trace, CGLS, finalize] device ms of the last phase-timed call."""
    buf = (ctypes.c_double * 3)()
    _check(load_library().mirage_last_phase_ms(ctx, buf), "mirage_last_phase_ms")
    return list(buf)


def mirage_eval_iter(ctx, probs, lens, prob_idx, n_iter=40, *, bhat=None, stream=None, real=torch.float32):
    """Fixed-iteration CGLS with the L-curve over iterations and, given ``bhat``
    (device tensor [n_probs, >= nx*ny] of the context's real type), the Monte
    Carlo degrees of freedom (mirage.h).  Returns a dict of device tensors."""
    lib = load_library()
    n = int(lens.shape[0])
    dev = lens.device
    max_ns = max(int(p.geom.sx) * int(p.geom.sy) for p in probs)
    pidx = np.ascontiguousarray(np.asarray(prob_idx, dtype=np.int32))
    mk = lambda shape, dt: torch.empty(shape, dtype=dt, device=dev)
    out = {"chi2": mk((n, n_iter + 1), torch.float64), "reg": mk((n, n_iter + 1), torch.float64),
           "kappa": mk((n, n_iter + 1), torch.float64), "corner": mk((n,), torch.int32),
           "s": mk((n, max_ns), real), "status": mk((n,), torch.int32)}
    stride = 0
    if bhat is not None:
        bhat = bhat.contiguous()
        stride = int(bhat.shape[-1])
        out["dof"] = mk((n, n_iter + 1), torch.float64)
    arr = (mirage_problem_t * len(probs))(*[p.c_struct() for p in probs])
    rc = lib.mirage_eval_iter(ctx, arr, len(probs), _ptr(lens.contiguous()), pidx.ctypes.data_as(ctypes.c_void_p), n,
                              int(n_iter), _ptr(bhat), stride, _ptr(out["chi2"]), _ptr(out["reg"]),
                              _ptr(out.get("dof")), _ptr(out["corner"]), _ptr(out["kappa"]), _ptr(out["s"]),
                              _ptr(out["status"]), _stream_ptr(stream))
    _check(rc, "mirage_eval_iter")
    return out


def mirage_measure_ffma(device=0):
    """(TFLOP/s, flops per clock per SM) the FP32 FMA pipe sustains (mirage.h)."""
    tf, fc = ctypes.c_double(), ctypes.c_double()
    _check(load_library().mirage_measure_ffma(int(device), ctypes.byref(tf), ctypes.byref(fc)), "mirage_measure_ffma")
    return tf.value, fc.value


def mirage_last_phase_clocks(ctx):
    """Per-phase SM clock totals of the last phase-clocked call (see mirage.h)."""
    buf = (ctypes.c_ulonglong * N_PHASE_CLOCKS)()
    _check(load_library().mirage_last_phase_clocks(ctx, buf), "mirage_last_phase_clocks")
    return list(buf)


def mirage_lcurve(chi2, reg, n_lam, *, stream=None):
    """Device L-curve corner of [n, max_lam] chi2/reg curves (n_lam device int32)."""
    lib = load_library()
    n, max_lam = int(chi2.shape[0]), int(chi2.shape[1])
    corner = torch.empty(n, dtype=torch.int32, device=chi2.device)
    kappa = torch.empty((n, max_lam), dtype=torch.float64, device=chi2.device)
    flags = torch.empty(n, dtype=torch.int32, device=chi2.device)
    _check(lib.mirage_lcurve(_ptr(chi2.contiguous()), _ptr(reg.contiguous()), _ptr(n_lam.contiguous()), n,
                             max_lam, _ptr(corner), _ptr(kappa), _ptr(flags), _stream_ptr(stream)),
           "mirage_lcurve")
    return corner, kappa, flags


def mirage_forward(ctx, prob, lens, S, *, want_model=True, stream=None):
    """B L s and chi2 for sources S [n_src, ns] at one lens (device tensors)."""
    lib = load_library()
    n_src = int(S.shape[0])
    model = torch.empty((n_src, int(prob.geom.ny) * int(prob.geom.nx)), dtype=S.dtype, device=S.device) \
        if want_model else None
    chi2 = torch.empty(n_src, dtype=torch.float64, device=S.device)
    status = torch.zeros(1, dtype=torch.int32, device=S.device)
    st = prob.c_struct()
    _check(lib.mirage_forward(ctx, ctypes.byref(st), _ptr(lens.contiguous()), _ptr(S.contiguous()), n_src,
                              _ptr(model), _ptr(chi2), _ptr(status), _stream_ptr(stream)), "mirage_forward")
    return model, chi2, status


def mirage_forward_noalloc(precision, prob, lens, S, *, want_model=True, stream=None):
    """B L s and chi2 like mirage_forward, without any device allocation by
    the library (all its scratch sits in a fixed array; see mirage.h).  The
    output tensors are allocated here by the caller-side binding."""
    lib = load_library()
    n_src = int(S.shape[0])
    model = torch.empty((n_src, int(prob.geom.ny) * int(prob.geom.nx)), dtype=S.dtype, device=S.device) \
        if want_model else None
    chi2 = torch.empty(n_src, dtype=torch.float64, device=S.device)
    status = torch.zeros(1, dtype=torch.int32, device=S.device)
    st = prob.c_struct()
    rc = lib.mirage_forward_noalloc(int(precision), ctypes.byref(st), _ptr(lens.contiguous()), _ptr(S.contiguous()),
                                    n_src, _ptr(model), _ptr(chi2), _ptr(status), _stream_ptr(stream))
    if rc != MIRAGE_OK:
        raise MirageError(f"mirage_forward_noalloc failed ({rc}): "
                          f"{lib.mirage_noalloc_last_error().decode(errors='replace')}")
    return model, chi2, status


def mirage_psf_blur(engine, img, psf, reps=1, *, out=None, stream=None):
    """B applied ``reps`` times to each image of ``img`` [n, ny, nx] (FP32,
    device) with the K x K ``psf`` (host array) on the FFMA or the
    tensor-core engine (see mirage.h).  Returns the output tensor."""
    lib = load_library()
    img = img.contiguous()
    n, ny, nx = (int(d) for d in img.shape)
    psf = np.ascontiguousarray(np.asarray(psf, dtype=np.float32))
    if out is None:
        out = torch.empty_like(img)
    rc = lib.mirage_psf_blur(int(engine), _ptr(img), _ptr(out), n, nx, ny, psf.ctypes.data_as(ctypes.c_void_p),
                             int(psf.shape[0]), int(reps), _stream_ptr(stream))
    if rc != MIRAGE_OK:
        raise MirageError(f"mirage_psf_blur failed ({rc}): {lib.mirage_blur_last_error().decode(errors='replace')}")
    return out


class MLP:
    """Surrogate network (see mirage.h): FP32 device tensors in and out."""

    def __init__(self, dims, device: int = 0, seed: int = 0):
        lib = load_library()
        self.dims = [int(d) for d in dims]
        arr = (ctypes.c_int * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        rc = lib.mirage_mlp_create(ctypes.byref(h), device, len(self.dims) - 1, arr, seed)
        self._chk(rc, "mirage_mlp_create")
        self.handle = h
        self.n_params = int(lib.mirage_mlp_num_params(h))

    @staticmethod
    def _chk(rc, what):
        if rc != MIRAGE_OK:
            raise MirageError(f"{what} failed ({rc}): {load_library().mirage_mlp_last_error().decode(errors='replace')}")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self._chk(load_library().mirage_mlp_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p),
                                                       self.n_params), "mirage_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        self._chk(load_library().mirage_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p), p.size),
                  "mirage_mlp_set_params")

    def layers(self, flat=None):
        """Split a flat parameter vector into [(W, b), ...]."""
        flat = self.get_params() if flat is None else flat
        out, o = [], 0
        for i, j in zip(self.dims[:-1], self.dims[1:]):
            W = flat[o:o + i * j].reshape(j, i)
            o += i * j
            b = flat[o:o + j]
            o += j
            out.append((W, b))
        return out

    def forward(self, x, stream=None):
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=torch.float32, device=x.device)
        self._chk(load_library().mirage_mlp_forward(self.handle, _ptr(x.contiguous()), int(x.shape[0]), _ptr(y),
                                                    _stream_ptr(stream)), "mirage_mlp_forward")
        return y

    def grad(self, x, t, stream=None):
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=torch.float32, device=x.device)
        self._chk(load_library().mirage_mlp_grad(self.handle, _ptr(x.contiguous()), _ptr(t.contiguous()),
                                                 int(x.shape[0]), _ptr(g), _ptr(loss), _ptr(y), _stream_ptr(stream)),
                  "mirage_mlp_grad")
        return g, loss, y

    def train(self, x, t, steps, batch, lr, seed=0, stream=None):
        """``steps`` Adam steps on minibatches of ``batch`` rows of (x, t)
        drawn on the device (mirage_mlp_train)."""
        x, t = x.contiguous(), t.contiguous()
        self._chk(load_library().mirage_mlp_train(self.handle, _ptr(x), _ptr(t), int(x.shape[0]), int(steps),
                                                  int(batch), float(lr), int(seed) & (2 ** 64 - 1),
                                                  _stream_ptr(stream)), "mirage_mlp_train")
        self._keep = (x, t)  # alive until the next call (the work is asynchronous)

    def train_step(self, x, t, lr, stream=None):
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=torch.float32, device=x.device)
        self._chk(load_library().mirage_mlp_train_step(self.handle, _ptr(x.contiguous()), _ptr(t.contiguous()),
                                                       int(x.shape[0]), float(lr), _ptr(loss), _ptr(y),
                                                       _stream_ptr(stream)), "mirage_mlp_train_step")
        return loss

    def close(self):
        if getattr(self, "handle", None) is not None:
            load_library().mirage_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owning wrapper of a mirage context (FP32 or FP64)."""

    def __init__(self, device: int = 0, precision: int = MIRAGE_FP32):
        self.precision = precision
        self.real = torch.float32 if precision == MIRAGE_FP32 else torch.float64
        self.device = device
        self.handle = mirage_create(device, precision)

    def eval_batch(self, probs, lens, prob_idx, lambdas, n_lam, **kw):
        kw.setdefault("real", self.real)
        return mirage_eval_batch(self.handle, probs, lens, prob_idx, lambdas, n_lam, **kw)

    def eval_iter(self, probs, lens, prob_idx, n_iter=40, **kw):
        kw.setdefault("real", self.real)
        return mirage_eval_iter(self.handle, probs, lens, prob_idx, n_iter, **kw)

    def forward(self, prob, lens, S, **kw):
        return mirage_forward(self.handle, prob, lens, S, **kw)

    def reserve_slots(self, slots: int):
        """Leave ``slots`` CTA slots free in the CGLS launches (mirage_set_reserved_slots)."""
        _check(load_library().mirage_set_reserved_slots(self.handle, int(slots)), "mirage_set_reserved_slots")

    def launches(self) -> int:
        return mirage_last_launch_count(self.handle)

    def phase_ms(self):
        return mirage_last_phase_ms(self.handle)

    def phase_clocks(self):
        return mirage_last_phase_clocks(self.handle)

    def close(self):
        if self.handle is not None:
            mirage_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
