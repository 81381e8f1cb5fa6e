"""Python binding of the GFK walker library (``include/gfk.h``), by ctypes.

Argument marshalling only: every step of the walk runs in the CUDA kernels of
``libgfk.so``.  The functions below carry the C names; ``Context`` wraps them
for convenience.  PyTorch is used only to hand the library the current CUDA
stream.  If the library cannot be built or loaded the import of any entry
point raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

# enums of include/gfk.h
GFK_OK, GFK_EINVAL, GFK_ENOMEM, GFK_ECUDA, GFK_ESTATE, GFK_ENONFINITE, GFK_EOVERFLOW, \
    GFK_ETIMEOUT = range(8)
GFK_1S, GFK_2S3, GFK_PZ = 0, 1, 2
GFK_PREC_FP64, GFK_PREC_MIXED = 0, 1
GFK_NOISE_GAUSSIAN, GFK_NOISE_BERNOULLI = 0, 1
GFK_TRIAL_JASTROW_PRODUCT, GFK_TRIAL_ORBITAL_PAIRS = 0, 1
GFK_MAX_TERMS = 4
GFK_MAX_INSTANCES = 64

# every entry point the header declares
EXPORTS = ("gfk_create", "gfk_set_trial", "gfk_set_launch", "gfk_propagate", "gfk_steps",
           "gfk_energy", "gfk_sums", "gfk_get_walkers", "gfk_counters", "gfk_checkpoint_size",
           "gfk_checkpoint", "gfk_restore", "gfk_profile", "gfk_profile_read", "gfk_reset",
           "gfk_destroy", "gfk_status_string", "gfk_last_error", "gfk_propagate_noalloc",
           "gfk_measure_peak", "gfk_set_graph", "gfk_autotune", "gfk_grad",
           "gfk_normal_moments", "gfk_kernel_count", "gfk_eval_f32", "gfk_debug_status")
PEAK_OPS = ("ffma", "dfma", "imad", "imad_hi", "imad_wide", "lop3", "ex2", "rsq", "lg2", "sin",
            "i2f", "f2f", "ffma2")
GFK_NOALLOC_SCRATCH_BYTES = 32 << 20
GFK_NOALLOC_MAX_WALKERS = 1 << 22


class gfk_instance_desc(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("n_walkers", ctypes.c_int64), ("dt", ctypes.c_double),
                ("e_trial", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("rng_stream", ctypes.c_uint32), ("ee_on", ctypes.c_int32),
                ("init_sigma", ctypes.c_double), ("walker_id0", ctypes.c_uint32),
                ("noise", ctypes.c_int32)]


class GfkError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libgfk.so (building it in-tree first if sources changed); with GFK_DEBUG=1 in
    the environment, the bounds-checked libgfk_debug.so instead (gfk_debug_status)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        debug = os.environ.get("GFK_DEBUG", "0") not in ("", "0")
        if debug:
            path = _build.build(debug=True) if build_if_needed else _build.LIB_DEBUG
        else:
            path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgfk.so missing at {path}; build it with "
                               "python -m paper_1703_08977_gb300.build")
        lib = ctypes.CDLL(path)
        c = ctypes
        P = c.c_void_p
        dp = c.POINTER(c.c_double)
        sig = {
            "gfk_create": ([c.POINTER(gfk_instance_desc), c.c_int32, P, c.POINTER(P)], c.c_int),
            "gfk_set_trial": ([P, c.c_int32, c.c_int32, dp, c.c_int32], c.c_int),
            "gfk_set_launch": ([P, c.c_int32, c.c_int32], c.c_int),
            "gfk_propagate": ([P, c.c_int64], c.c_int),
            "gfk_steps": ([P, c.POINTER(c.c_int64)], c.c_int),
            "gfk_energy": ([P, c.c_int32, dp, dp, dp, c.c_int64, dp], c.c_int),
            "gfk_sums": ([P, c.c_int32, dp, c.c_int64], c.c_int),
            "gfk_get_walkers": ([P, c.c_int32, dp, dp, c.POINTER(c.c_uint8)], c.c_int),
            "gfk_counters": ([P, c.c_int32, c.POINTER(c.c_int64)], c.c_int),
            "gfk_checkpoint_size": ([P, c.POINTER(c.c_int64)], c.c_int),
            "gfk_checkpoint": ([P, P, c.c_int64], c.c_int),
            "gfk_restore": ([P, P, c.c_int64], c.c_int),
            "gfk_profile": ([P, c.c_int32], c.c_int),
            "gfk_profile_read": ([P, dp, c.POINTER(c.c_int64), dp, c.c_int32], c.c_int),
            "gfk_reset": ([P], c.c_int),
            "gfk_destroy": ([P], None),
            "gfk_status_string": ([c.c_int], c.c_char_p),
            "gfk_last_error": ([P], c.c_char_p),
            "gfk_measure_peak": ([c.c_int32, P, dp], c.c_int),
            "gfk_normal_moments": ([c.c_int32, P, dp], c.c_int),
            "gfk_kernel_count": ([P, c.POINTER(c.c_int64), c.c_int32], c.c_int),
            "gfk_eval_f32": ([c.c_int32, dp, c.c_int32, c.c_int32, c.c_int64,
                              c.POINTER(c.c_float), c.c_int32, c.POINTER(c.c_float),
                              c.POINTER(c.c_float), c.POINTER(c.c_int32), P], c.c_int),
            "gfk_set_graph": ([P, c.c_int32], c.c_int),
            "gfk_grad": ([P, c.c_int32, c.c_int32, c.c_int64, c.c_int32, dp, c.c_int32, dp],
                         c.c_int),
            "gfk_autotune": ([P, c.c_int64, c.POINTER(c.c_int32), c.POINTER(c.c_int32), dp],
                             c.c_int),
            "gfk_propagate_noalloc": ([c.POINTER(gfk_instance_desc), c.c_int32, dp, c.c_int32,
                                       P, P, P, c.c_int32, c.c_int64, c.c_int64, P, P, P],
                                      c.c_int),
            "gfk_debug_status": ([c.POINTER(c.c_int32), c.POINTER(c.c_uint32),
                                  c.POINTER(c.c_uint64), c.c_int32], c.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def status_string(status: int) -> str:
    return load().gfk_status_string(int(status)).decode()


def gfk_status_string(status: int) -> str:
    return status_string(status)


def gfk_last_error(ctx) -> str:
    return load().gfk_last_error(ctx).decode()


def _check(status, where, ctx=None, ok=(GFK_OK,)):
    if status not in ok:
        raise GfkError(status, where, gfk_last_error(ctx) if ctx else "")
    return status


def _current_stream_ptr():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the GFK library needs a CUDA GPU")
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------------------
# Entry points with the C names (host arrays are numpy).
# ----------------------------------------------------------------------------
def gfk_create(descs, stream=None):
    """descs: sequence of gfk_instance_desc (or InstanceDesc); returns the ctx handle."""
    lib = load()
    arr = (gfk_instance_desc * len(descs))(*[d.c() if isinstance(d, InstanceDesc) else d
                                             for d in descs])
    if stream is None:
        stream = _current_stream_ptr()
    out = ctypes.c_void_p()
    _check(lib.gfk_create(arr, len(descs), stream, ctypes.byref(out)), "gfk_create")
    return out


def gfk_set_trial(ctx, inst, kind, params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(load().gfk_set_trial(ctx, int(inst), int(kind), _dp(p), len(p)), "gfk_set_trial", ctx)


def gfk_set_launch(ctx, threads_per_block, walkers_per_thread):
    _check(load().gfk_set_launch(ctx, int(threads_per_block), int(walkers_per_thread)),
           "gfk_set_launch", ctx)


def gfk_propagate(ctx, n_steps):
    _check(load().gfk_propagate(ctx, int(n_steps)), "gfk_propagate", ctx)


def gfk_steps(ctx) -> int:
    v = ctypes.c_int64()
    _check(load().gfk_steps(ctx, ctypes.byref(v)), "gfk_steps", ctx)
    return v.value


def gfk_energy(ctx, inst, cap=None, out=None):
    """Returns (e_mixed, ln_z, ess, e_final, status); status may be GFK_ENONFINITE."""
    n = gfk_steps(ctx) + 1
    cap = n if cap is None else int(cap)
    if out is None:
        e, lz, es = np.empty(cap), np.empty(cap), np.empty(cap)
    else:
        e, lz, es = out
    ef = ctypes.c_double()
    st = load().gfk_energy(ctx, int(inst), _dp(e), _dp(lz), _dp(es), cap, ctypes.byref(ef))
    _check(st, "gfk_energy", ctx, ok=(GFK_OK, GFK_ENONFINITE))
    return e[:n], lz[:n], es[:n], ef.value, st


def gfk_sums(ctx, inst):
    n = gfk_steps(ctx) + 1
    rows = np.empty((n, 6))
    _check(load().gfk_sums(ctx, int(inst), _dp(rows), n), "gfk_sums", ctx)
    return rows


def gfk_get_walkers(ctx, inst, n_walkers):
    x = np.empty((int(n_walkers), 6))
    lw = np.empty(int(n_walkers))
    al = np.empty(int(n_walkers), dtype=np.uint8)
    _check(load().gfk_get_walkers(ctx, int(inst), _dp(x), _dp(lw),
                                  al.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
           "gfk_get_walkers", ctx)
    return x, lw, al


def gfk_counters(ctx, inst):
    c = np.zeros(3, dtype=np.int64)
    _check(load().gfk_counters(ctx, int(inst), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "gfk_counters", ctx)
    return c


def gfk_checkpoint_size(ctx) -> int:
    v = ctypes.c_int64()
    _check(load().gfk_checkpoint_size(ctx, ctypes.byref(v)), "gfk_checkpoint_size", ctx)
    return v.value


def gfk_checkpoint(ctx) -> bytes:
    n = gfk_checkpoint_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load().gfk_checkpoint(ctx, ctypes.cast(buf, ctypes.c_void_p), n), "gfk_checkpoint", ctx)
    return buf.raw


def gfk_restore(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().gfk_restore(ctx, ctypes.cast(buf, ctypes.c_void_p), len(blob)), "gfk_restore", ctx)


def gfk_profile(ctx, enable=True):
    _check(load().gfk_profile(ctx, int(bool(enable))), "gfk_profile", ctx)


def gfk_profile_read(ctx, reset=True):
    """(summed walk-kernel ms, launches, walker-steps) since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    ws = ctypes.c_double()
    _check(load().gfk_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(ws),
                                   int(bool(reset))), "gfk_profile_read", ctx)
    return ms.value, n.value, ws.value


def gfk_kernel_count(ctx, reset=False) -> int:
    """Kernels gfk_propagate has queued since creation or the last reset of the count."""
    v = ctypes.c_int64()
    _check(load().gfk_kernel_count(ctx, ctypes.byref(v), int(bool(reset))), "gfk_kernel_count")
    return int(v.value)


def gfk_reset(ctx):
    _check(load().gfk_reset(ctx), "gfk_reset", ctx)


def gfk_destroy(ctx):
    load().gfk_destroy(ctx)


def gfk_propagate_noalloc(desc, kind, params, p0, p1, sgn, init, step0, n_steps, rows, counters,
                          stream=None):
    """Allocation-free mixed walk on caller-provided device buffers (torch CUDA tensors:
    p0, p1 float32 (n, 4); sgn int8 (n,); rows float64 (n_steps + init, 6); counters
    int64 (3,)).  Passes their device addresses through unchanged; returns the status."""
    d = desc.c() if isinstance(desc, InstanceDesc) else desc
    p = np.ascontiguousarray(params, dtype=np.float64)
    if stream is None:
        stream = _current_stream_ptr()
    addr = lambda t: ctypes.c_void_p(t.data_ptr())
    return load().gfk_propagate_noalloc(ctypes.byref(d), int(kind), _dp(p), len(p), addr(p0),
                                        addr(p1), addr(sgn), int(init), int(step0),
                                        int(n_steps), addr(rows), addr(counters), stream)


def gfk_grad(ctx, inst, loss_kind, n_steps, ckpt_every=64):
    """(loss, gradient over [Z, a, beta, c1, c2, c3, c4]) of instance inst's walk."""
    g = np.zeros(7)
    l = ctypes.c_double()
    _check(load().gfk_grad(ctx, int(inst), int(loss_kind), int(n_steps), int(ckpt_every), _dp(g),
                           7, ctypes.byref(l)), "gfk_grad", ctx)
    return l.value, g


def gfk_debug_status(clear=True):
    """(debug_build, flags, first_addr) of the debug build's bounds checks (zeros in the
    release build); clears them when `clear`."""
    b, f, a = ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_uint64()
    _check(load().gfk_debug_status(ctypes.byref(b), ctypes.byref(f), ctypes.byref(a),
                                   int(bool(clear))), "gfk_debug_status")
    return b.value, f.value, a.value


def gfk_set_graph(ctx, enable=True):
    _check(load().gfk_set_graph(ctx, int(bool(enable))), "gfk_set_graph", ctx)


def gfk_autotune(ctx, probe_steps=256):
    """(threads, walkers_per_thread, walker-steps/s) of the fastest launch shape; applied."""
    t = ctypes.c_int32()
    w = ctypes.c_int32()
    r = ctypes.c_double()
    _check(load().gfk_autotune(ctx, int(probe_steps), ctypes.byref(t), ctypes.byref(w),
                               ctypes.byref(r)), "gfk_autotune", ctx)
    return t.value, w.value, r.value


def autotune_cached(ctx, descs, trials, probe_steps=256, path=None):
    """gfk_autotune with a JSON cache keyed by device, precision, noise mode, trial kinds
    and walker counts (in the package's build folder); a cached shape is applied without
    timing."""
    import json
    import torch
    path = path or os.path.join(os.path.dirname(_build.LIB), "autotune.json")
    key = json.dumps({"device": torch.cuda.get_device_name(),
                      "prec": int(descs[0].prec), "noise": int(descs[0].noise),
                      "kinds": [int(k) for k, _ in trials],
                      "walkers": [int(d.n_walkers) for d in descs]}, sort_keys=True)
    cache = {}
    if os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        t, w, r = cache[key]
        gfk_set_launch(ctx, t, w)
        return t, w, r
    t, w, r = gfk_autotune(ctx, probe_steps)
    cache[key] = [t, w, r]
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, path)
    return t, w, r


def gfk_measure_peak(op, stream=None) -> float:
    """Measured lane-operations per second of one instruction class (see PEAK_OPS)."""
    if isinstance(op, str):
        op = PEAK_OPS.index(op)
    if stream is None:
        stream = _current_stream_ptr()
    v = ctypes.c_double()
    _check(load().gfk_measure_peak(int(op), stream, ctypes.byref(v)), "gfk_measure_peak")
    return v.value


def gfk_eval_f32(kind, params, x, lanes=2, ee_on=1, stream=None):
    """The mixed walk's FP32 trial evaluation at positions x (n, 6): (b (n, 6) float32,
    E_L (n,) float32, sign (n,) int32)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xv = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 6)
    n = xv.shape[0]
    b = np.empty((n, 6), dtype=np.float32)
    el = np.empty(n, dtype=np.float32)
    sg = np.empty(n, dtype=np.int32)
    if stream is None:
        stream = _current_stream_ptr()
    fp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    _check(load().gfk_eval_f32(int(kind), _dp(p), len(p), int(ee_on), n, fp(xv), int(lanes),
                               fp(b), fp(el), sg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               stream), "gfk_eval_f32")
    return b, el, sg


RADIUS_METHODS = ("kernel", "hw_log2", "logf")


MOMENT_NAMES = ("r2_err", "rho2_err", "cos2_err", "sin2_err", "cos_mean", "sin_mean")


def gfk_normal_moments(method="kernel", stream=None) -> dict:
    """Exhaustive moments of the FP32 Box-Muller normals against FP64 (see gfk.h)."""
    if isinstance(method, str):
        method = RADIUS_METHODS.index(method)
    if stream is None:
        stream = _current_stream_ptr()
    v = (ctypes.c_double * 6)()
    _check(load().gfk_normal_moments(int(method), stream, v), "gfk_normal_moments")
    return dict(zip(MOMENT_NAMES, list(v)))


# ----------------------------------------------------------------------------
# Convenience wrapper
# ----------------------------------------------------------------------------
@dataclass
class InstanceDesc:
    n_walkers: int
    dt: float
    e_trial: float
    seed: int = 0
    state: int = GFK_1S
    prec: int = GFK_PREC_FP64
    rng_stream: int = 0
    ee_on: int = 1
    init_sigma: float = 0.5
    walker_id0: int = 0
    noise: int = GFK_NOISE_GAUSSIAN

    def c(self) -> gfk_instance_desc:
        return gfk_instance_desc(int(self.state), int(self.prec), int(self.n_walkers),
                                 float(self.dt), float(self.e_trial), int(self.seed),
                                 int(self.rng_stream), int(self.ee_on), float(self.init_sigma),
                                 int(self.walker_id0), int(self.noise))


class Context:
    """Owns one gfk_ctx; instances are described by InstanceDesc."""

    def __init__(self, descs, trials=None, stream=None, launch=None):
        self.descs = list(descs)
        self.handle = gfk_create(self.descs, stream)
        if trials is not None:
            for i, (kind, params) in enumerate(trials):
                gfk_set_trial(self.handle, i, kind, params)
        if launch is not None:
            gfk_set_launch(self.handle, *launch)

    def set_trial(self, inst, kind, params):
        gfk_set_trial(self.handle, inst, kind, params)

    def set_launch(self, threads, wpt):
        gfk_set_launch(self.handle, threads, wpt)

    def set_graph(self, enable=True):
        gfk_set_graph(self.handle, enable)

    def autotune(self, probe_steps=256, cache=True, trials=None):
        if cache:
            return autotune_cached(self.handle, self.descs, trials or [(0, None)] * len(self.descs),
                                   probe_steps)
        return gfk_autotune(self.handle, probe_steps)

    def propagate(self, n_steps):
        gfk_propagate(self.handle, n_steps)
        return self

    @property
    def steps(self):
        return gfk_steps(self.handle)

    def energy(self, inst=0):
        e, lz, es, ef, st = gfk_energy(self.handle, inst)
        return {"E": e, "ln_z": lz, "ess": es, "e_final": ef, "status": st}

    def sums(self, inst=0):
        return gfk_sums(self.handle, inst)

    def walkers(self, inst=0):
        return gfk_get_walkers(self.handle, inst, self.descs[inst].n_walkers)

    def counters(self, inst=0):
        return gfk_counters(self.handle, inst)

    def checkpoint(self):
        return gfk_checkpoint(self.handle)

    def restore(self, blob):
        gfk_restore(self.handle, blob)

    def reset(self):
        gfk_reset(self.handle)

    def close(self):
        if self.handle is not None:
            gfk_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
