"""Thin ctypes binding of include/ffe.h (argument marshalling only).

Every function of the C ABI is exposed under its own name; numpy structured
arrays with the C layouts carry the batches.  No arithmetic of the method
happens here: the CUDA library does all of it, and importing this module
never falls back to anything else -- if libffe.so is missing or cannot be
loaded the calls raise FFEError.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffe.so")

FFE_OK, FFE_EINVAL, FFE_ENOMEM, FFE_ECUDA, FFE_ETIMEOUT, FFE_EUNSUPPORTED, FFE_EINTERNAL = range(7)
FFE_FP64, FFE_FP32C = 0, 1
FFE_MODEL_RAGHU2, FFE_MODEL_DAGHOFER3 = 0, 1

# Printed model parameters: App. A (two-band, units of |t1|) and App. B
# (three-band, eV; n = 4 at mu = 0.4748).
RAGHU2_PARAMS = dict(t1=-1.0, t2=1.3, t3=-0.85, t4=-0.85, mu=1.54)
DAGHOFER3_PARAMS = dict(t1=-0.08, t2=0.1825, t3=0.08375, t4=-0.03, t5=0.15, t6=0.15, t7=-0.12, t8=0.06,
                        t9=0.0, t10=-0.024, t11=-0.01, t12=0.0275, eps0=0.75, mu=0.4748)
MODELS = {"raghu2": (FFE_MODEL_RAGHU2, 2, RAGHU2_PARAMS), "daghofer3": (FFE_MODEL_DAGHOFER3, 3, DAGHOFER3_PARAMS)}
FFE_SEARCH_GRID, FFE_SEARCH_GOLDEN = 0, 1
FFE_FLAG_RESCORED, FFE_FLAG_EDGE, FFE_FLAG_LOWER, FFE_FLAG_PRUNED, FFE_FLAG_INVALID = 1, 2, 4, 8, 32
FFE_PHASE_NORMAL, FFE_PHASE_BCS, FFE_PHASE_FFLO = 0, 1, 2

POINT_DTYPE = np.dtype([("N", "<i4"), ("reserved", "<i4"), ("qx", "<f8"), ("qy", "<f8"),
                        ("h", "<f8"), ("T", "<f8"), ("delta", "<f8")])
PARAM_DTYPE = np.dtype([("N", "<i4"), ("n", "<i4"), ("qx", "<f8"), ("qy", "<f8"), ("h", "<f8"),
                        ("T", "<f8"), ("lo", "<f8"), ("hi", "<f8")])
RESULT_DTYPE = np.dtype([("delta_star", "<f8"), ("omega_star", "<f8"), ("omega_lo", "<f8"),
                         ("err_bound", "<f8"), ("idx_star", "<i4"), ("flags", "<i4")])


class FFEError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        super().__init__(f"ffe status {status}: {message}")


class ffe_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("prec", ctypes.c_int32), ("t1", ctypes.c_double),
                ("t2", ctypes.c_double), ("t3", ctypes.c_double), ("t4", ctypes.c_double),
                ("mu", ctypes.c_double), ("U", ctypes.c_double), ("eta_amp", ctypes.c_double)] + [
                    (f"t{i}", ctypes.c_double) for i in range(5, 13)] + [("eps0", ctypes.c_double),
                                                                         ("U_band", ctypes.c_double * 3)]


class ffe_scan(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("n_q", ctypes.c_int32),
                ("qx", ctypes.POINTER(ctypes.c_double)), ("qy", ctypes.POINTER(ctypes.c_double)),
                ("n_h", ctypes.c_int32), ("n_T", ctypes.c_int32),
                ("h", ctypes.POINTER(ctypes.c_double)), ("T", ctypes.POINTER(ctypes.c_double)),
                ("search", ctypes.c_int32), ("n", ctypes.c_int32),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double)]


class ffe_plan_info(ctypes.Structure):
    _fields_ = [("k_evals", ctypes.c_double), ("device_bytes", ctypes.c_double), ("launches", ctypes.c_int32),
                ("rescored_search", ctypes.c_int32), ("rescored_labels", ctypes.c_int32),
                ("kpt", ctypes.c_int32), ("block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("work_items", ctypes.c_int32), ("reserved", ctypes.c_int32), ("k_evals_near", ctypes.c_double),
                ("k_evals_single", ctypes.c_double), ("k_evals_far_closed", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/ffe.h
_VP = ctypes.c_void_p
_SIGNATURES = [
    ("ffe_create", ctypes.c_int, [ctypes.POINTER(ffe_model), ctypes.POINTER(_VP)]),
    ("ffe_destroy", None, [_VP]),
    ("ffe_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ffe_last_error", ctypes.c_char_p, [_VP]),
    ("ffe_omega", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    ("ffe_minimize", ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP]),
    ("ffe_minimize_bands", ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, _VP]),
    ("ffe_pair_susceptibility", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, ctypes.c_double,
                                               ctypes.c_double, _VP, _VP]),
    ("ffe_phase_scan", ctypes.c_int, [_VP, ctypes.POINTER(ffe_scan), _VP, _VP, _VP, _VP]),
    ("ffe_plan_phase_scan", ctypes.c_int, [_VP, ctypes.POINTER(ffe_scan), _VP, ctypes.POINTER(_VP)]),
    ("ffe_plan_execute", ctypes.c_int, [_VP, _VP]),
    ("ffe_plan_fetch", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("ffe_plan_stats", ctypes.c_int, [_VP, ctypes.POINTER(ffe_plan_info)]),
    ("ffe_plan_fetch_grid", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("ffe_plan_kernel_ms", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    ("ffe_plan_destroy", None, [_VP]),
    ("ffe_plan_minimize", ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.POINTER(_VP)]),
    ("ffe_plan_fetch_minimize", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("ffe_plan_autotune", ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]),
    ("ffe_probe_peaks", ctypes.c_int, [_VP]),
    ("ffe_surrogate_create", ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(_VP)]),
    ("ffe_surrogate_destroy", None, [_VP]),
    ("ffe_surrogate_set_params", ctypes.c_int, [_VP, _VP]),
    ("ffe_surrogate_get_params", ctypes.c_int, [_VP, _VP]),
    ("ffe_surrogate_targets", ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _VP]),
    ("ffe_surrogate_predict", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("ffe_surrogate_save", ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("ffe_surrogate_load", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("ffe_surrogate_grad", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    ("ffe_surrogate_train", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_float, _VP, _VP]),
    ("ffe_surrogate_train_schedule", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                    _VP, _VP, _VP]),
    ("ffe_surrogate_scan", ctypes.c_int, [_VP, _VP, ctypes.POINTER(ffe_scan), _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ffe_omega_noalloc", ctypes.c_int, [ctypes.POINTER(ffe_model), ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP]),
    ("ffe_omega_async", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP,
                                       ctypes.c_int64, _VP, _VP, _VP]),
    ("ffe_minimize_async", ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    ("ffe_phase_scan_async", ctypes.c_int, [_VP, ctypes.POINTER(ffe_scan), _VP, _VP, _VP, _VP]),
    ("ffe_label_candidates", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    ("ffe_merge_candidates", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32, _VP,
                                            _VP]),
]


class ffe_guide(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("q_keep", ctypes.c_int32), ("margin", ctypes.c_double)]


class ffe_guide_stats(ctypes.Structure):
    _fields_ = [("k_evals", ctypes.c_double), ("k_evals_full", ctypes.c_double), ("lines_kept", ctypes.c_int64),
                ("lines_pruned", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("rms_error", ctypes.c_double),
                ("mlp_flops", ctypes.c_double)]


def ffe_surrogate_scan(ctx, sur, N, qx, qy, h, T, n=256, lo=0.0, hi=0.2, window=16, q_keep=3, stream=None,
                       search=FFE_SEARCH_GRID, margin=0.0):
    """Guided scan (grid: n points; golden: n reductions); returns (per_point, labels, best_q, stats dict)."""
    sc, keep = make_scan(N, qx, qy, h, T, search, n, lo, hi)
    npts = sc.n_h * sc.n_T
    res = np.zeros((sc.n_q, npts), dtype=RESULT_DTYPE)
    labels = np.zeros(npts, dtype=np.int8)
    best = np.zeros(npts, dtype=np.int32)
    g = ffe_guide(window, q_keep, float(margin))
    st = ffe_guide_stats()
    _check(ctx, lib().ffe_surrogate_scan(ctx, sur.handle, ctypes.byref(sc), ctypes.byref(g), _ptr(res),
                                         _ptr(labels), _ptr(best), ctypes.byref(st), _stream(stream)))
    del keep
    return res, labels, best, {name: getattr(st, name) for name, _ in ffe_guide_stats._fields_}

N_SURROGATE_PARAMS = 33793


class ffe_surrogate_meta(ctypes.Structure):
    _fields_ = [("shift", ctypes.c_float * 4), ("scale", ctypes.c_float * 4), ("y_scale", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class Surrogate:
    """Owning wrapper of an ffe_surrogate (the learned proposal model)."""

    def __init__(self, ctx: "Context", shift, scale, y_scale, params=None):
        meta = ffe_surrogate_meta((ctypes.c_float * 4)(*shift), (ctypes.c_float * 4)(*scale), float(y_scale), 0)
        self.ctx = ctx
        self.handle = _VP()
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        _check(ctx.handle, lib().ffe_surrogate_create(ctx.handle, ctypes.byref(meta), _ptr(p), ctypes.byref(self.handle)))

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(self.ctx.handle, lib().ffe_surrogate_set_params(self.handle, _ptr(p)))

    def get_params(self):
        p = np.zeros(N_SURROGATE_PARAMS, dtype=np.float32)
        _check(self.ctx.handle, lib().ffe_surrogate_get_params(self.handle, _ptr(p)))
        return p

    def save(self) -> bytes:
        """Checkpoint (weights, Adam moments and step, input/output maps) as bytes."""
        n = ctypes.c_size_t(0)
        _check(self.ctx.handle, lib().ffe_surrogate_save(self.handle, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.ctx.handle, lib().ffe_surrogate_save(self.handle, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, data: bytes):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(self.ctx.handle, lib().ffe_surrogate_load(self.handle, buf, len(data)))

    def predict(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        y = np.zeros(len(x), dtype=np.float32)
        _check(self.ctx.handle, lib().ffe_surrogate_predict(self.handle, _ptr(x), len(x), _ptr(y), None))
        return y

    def grad(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(N_SURROGATE_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self.ctx.handle, lib().ffe_surrogate_grad(self.handle, _ptr(x), _ptr(t), len(x), _ptr(g),
                                                         ctypes.byref(loss), None))
        return loss.value, g

    def train(self, x, t, epochs, batch, lr):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, dtype=np.float32)
        losses = np.zeros(epochs, dtype=np.float32)
        _check(self.ctx.handle, lib().ffe_surrogate_train(self.handle, _ptr(x), _ptr(t), len(x), epochs, batch,
                                                          float(lr), _ptr(losses), None))
        return losses

    def train_schedule(self, x, t, lr_per_epoch, batch):
        """Training with one learning rate per epoch; the samples are uploaded once."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, dtype=np.float32)
        lrs = np.ascontiguousarray(lr_per_epoch, dtype=np.float32)
        losses = np.zeros(len(lrs), dtype=np.float32)
        _check(self.ctx.handle, lib().ffe_surrogate_train_schedule(self.handle, _ptr(x), _ptr(t), len(x), len(lrs),
                                                                   batch, _ptr(lrs), _ptr(losses), None))
        return losses

    def close(self):
        if self.handle:
            lib().ffe_surrogate_destroy(self.handle)
            self.handle = None


class ffe_peaks(ctypes.Structure):
    _fields_ = [("ex2", ctypes.c_double), ("lg2", ctypes.c_double), ("rsqrt", ctypes.c_double),
                ("rcp", ctypes.c_double), ("fma32", ctypes.c_double), ("fma64", ctypes.c_double),
                ("n_sm", ctypes.c_int32), ("sm_khz_max", ctypes.c_int32)]


def ffe_probe_peaks() -> dict:
    p = ffe_peaks()
    st = lib().ffe_probe_peaks(ctypes.byref(p))
    if st != FFE_OK:
        raise FFEError(st, lib().ffe_status_string(st).decode())
    return {name: getattr(p, name) for name, _ in ffe_peaks._fields_}


def lib():
    """Load libffe.so from the package directory (raises FFEError if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FFEError(FFE_EINTERNAL, f"{LIB_PATH} is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return [s[0] for s in _SIGNATURES]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_VP)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(ctx, st):
    if st != FFE_OK:
        msg = lib().ffe_last_error(ctx).decode() if ctx else ""
        if not msg:
            msg = lib().ffe_status_string(st).decode()
        raise FFEError(st, msg)


# ------------------------------------------------------------ entry points
def ffe_surrogate_targets(ctx, omega, N):
    """Condensation energies per site (omega[l, j] - omega[l, 0]) / N^2 in FP32 of the lines
    (rows) of omega, computed by the library."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    lines = om.reshape(-1, om.shape[-1])
    y = np.zeros(lines.shape, dtype=np.float32)
    _check(ctx, lib().ffe_surrogate_targets(ctx, _ptr(lines), lines.shape[0], lines.shape[1], int(N), _ptr(y)))
    return y.reshape(om.shape)


def ffe_create(U=2.0, eta_amp=1.0, prec=FFE_FP32C, model="raghu2", U_band=None, **params):
    """A context for `model` ("raghu2": App. A, "daghofer3": App. B) with its printed
    parameters, any of which `params` overrides; U_band: per-band couplings (0 = U)."""
    kind, _, defaults = MODELS[model]
    p = dict(defaults)
    p.update(params)
    ub = list(U_band or ()) + [0.0] * (3 - len(U_band or ()))
    m = ffe_model(kind=kind, prec=prec, U=U, eta_amp=eta_amp, U_band=(ctypes.c_double * 3)(*ub), **p)
    h = _VP()
    st = lib().ffe_create(ctypes.byref(m), ctypes.byref(h))
    if st != FFE_OK:
        raise FFEError(st, lib().ffe_status_string(st).decode())
    return h


def ffe_destroy(ctx):
    lib().ffe_destroy(ctx)


def ffe_omega(ctx, points: np.ndarray, stream=None, bands=0):
    """Omega at the points; with bands = nb (the model's band count) returns
    (omega[n], omega_band[n, nb])."""
    pts = np.ascontiguousarray(points, dtype=POINT_DTYPE)
    out = np.zeros(len(pts))
    ob = np.zeros((len(pts), int(bands))) if bands else None
    _check(ctx, lib().ffe_omega(ctx, _ptr(pts), len(pts), _ptr(out), _ptr(ob), _stream(stream)))
    return (out, ob) if bands else out


def ffe_minimize_bands(ctx, params: np.ndarray, search=FFE_SEARCH_GRID, stream=None, nb=2):
    """Per-band independent searches; returns results[n, nb] (bands ascending)."""
    ps = np.ascontiguousarray(params, dtype=PARAM_DTYPE)
    res = np.zeros((len(ps), nb), dtype=RESULT_DTYPE)
    _check(ctx, lib().ffe_minimize_bands(ctx, search, _ptr(ps), len(ps), _ptr(res), _stream(stream)))
    return res


def ffe_pair_susceptibility(ctx, N, qx, qy, h, T, nb=2, stream=None):
    """chi[n_q, nb, nb] of App. C at the pair momenta (qx[i], qy[i])."""
    qx = np.ascontiguousarray(np.atleast_1d(qx), dtype=np.float64)
    qy = np.ascontiguousarray(np.broadcast_to(np.asarray(qy, dtype=np.float64), qx.shape))
    out = np.zeros((len(qx), nb, nb))
    _check(ctx, lib().ffe_pair_susceptibility(ctx, int(N), len(qx), _ptr(qx), _ptr(qy), float(h), float(T),
                                              _ptr(out), _stream(stream)))
    return out


def ffe_minimize(ctx, params: np.ndarray, search=FFE_SEARCH_GRID, want_grid=False, stream=None):
    ps = np.ascontiguousarray(params, dtype=PARAM_DTYPE)
    res = np.zeros(len(ps), dtype=RESULT_DTYPE)
    grid = np.zeros(int(ps["n"].sum())) if want_grid else None
    err = np.zeros(int(ps["n"].sum())) if want_grid else None
    _check(ctx, lib().ffe_minimize(ctx, search, _ptr(ps), len(ps), _ptr(res), _ptr(grid), _ptr(err),
                                   _stream(stream)))
    return (res, grid, err) if want_grid else res


def _dptr(t):
    """Device address of a tensor-like argument (anything with data_ptr()), or None."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def ffe_omega_async(ctx, N, qx, qy, h, T, delta, omega, omega_band=None, stream=None):
    """Stream-ordered Omega at the points of one (N, Q): h, T, delta, omega (and omega_band,
    [n, nb]) are device tensors of float64; returns without waiting for the device."""
    _check(ctx, lib().ffe_omega_async(ctx, int(N), float(qx), float(qy), _dptr(h), _dptr(T), _dptr(delta),
                                      int(h.numel()), _dptr(omega), _dptr(omega_band), _stream(stream)))


def ffe_minimize_async(ctx, params: np.ndarray, out, search=FFE_SEARCH_GRID, omega_grid=None, stream=None):
    """Stream-ordered minimisation: params host (PARAM_DTYPE), out a device buffer of
    len(params) * RESULT_DTYPE.itemsize bytes (see result_buffer), omega_grid a device tensor."""
    ps = np.ascontiguousarray(params, dtype=PARAM_DTYPE)
    _check(ctx, lib().ffe_minimize_async(ctx, search, _ptr(ps), len(ps), _dptr(out), _dptr(omega_grid),
                                         _stream(stream)))


def ffe_phase_scan_async(ctx, N, qx, qy, h, T, per_point=None, labels=None, best_q=None, search=FFE_SEARCH_GRID,
                         n=256, lo=0.0, hi=0.2, stream=None):
    """Stream-ordered phase scan: per_point (result buffer), labels (int8) and best_q (int32)
    are device tensors or None."""
    sc, keep = make_scan(N, qx, qy, h, T, search, n, lo, hi)
    _check(ctx, lib().ffe_phase_scan_async(ctx, ctypes.byref(sc), _dptr(per_point), _dptr(labels), _dptr(best_q),
                                           _stream(stream)))
    del keep


def result_buffer(n, device="cuda"):
    """A device buffer for n ffe_result records (torch uint8); view it on the host with
    as_results(buffer)."""
    import torch

    return torch.empty(int(n) * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)


def as_results(buf) -> np.ndarray:
    return buf.cpu().numpy().view(RESULT_DTYPE)


def make_scan(N, qx, qy, h, T, search=FFE_SEARCH_GRID, n=256, lo=0.0, hi=0.2):
    """Returns (ffe_scan, keepalive arrays)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (qx, qy, h, T)]
    dp = ctypes.POINTER(ctypes.c_double)
    sc = ffe_scan(N, len(arrs[0]), arrs[0].ctypes.data_as(dp), arrs[1].ctypes.data_as(dp),
                  len(arrs[2]), len(arrs[3]), arrs[2].ctypes.data_as(dp), arrs[3].ctypes.data_as(dp),
                  search, n, lo, hi)
    return sc, arrs


def ffe_phase_scan(ctx, N, qx, qy, h, T, search=FFE_SEARCH_GRID, n=256, lo=0.0, hi=0.2, stream=None,
                   labels=True):
    """Returns (per_point[n_q, n_h*n_T], labels[n_h*n_T], best_q[n_h*n_T]); labels=False (a q
    list without Q = 0): the labels and best q are None."""
    sc, keep = make_scan(N, qx, qy, h, T, search, n, lo, hi)
    npts = sc.n_h * sc.n_T
    res = np.zeros((sc.n_q, npts), dtype=RESULT_DTYPE)
    labels = np.zeros(npts, dtype=np.int8) if labels else None
    best = np.zeros(npts, dtype=np.int32) if labels is not None else None
    _check(ctx, lib().ffe_phase_scan(ctx, ctypes.byref(sc), _ptr(res), _ptr(labels), _ptr(best),
                                     _stream(stream)))
    del keep
    return res, labels, best


def ffe_plan_phase_scan(ctx, N, qx, qy, h, T, search=FFE_SEARCH_GRID, n=256, lo=0.0, hi=0.2, stream=None):
    sc, keep = make_scan(N, qx, qy, h, T, search, n, lo, hi)
    plan = _VP()
    _check(ctx, lib().ffe_plan_phase_scan(ctx, ctypes.byref(sc), _stream(stream), ctypes.byref(plan)))
    del keep
    return Plan(ctx, plan, sc.n_q, sc.n_h * sc.n_T)


def ffe_plan_execute(plan, stream=None):
    _check(plan.ctx, lib().ffe_plan_execute(plan.handle, _stream(stream)))


def ffe_plan_fetch(plan, stream=None, labels=True):
    res = np.zeros((plan.n_q, plan.n_pts), dtype=RESULT_DTYPE)
    labels = np.zeros(plan.n_pts, dtype=np.int8) if labels else None
    best = np.zeros(plan.n_pts, dtype=np.int32) if labels is not None else None
    _check(plan.ctx, lib().ffe_plan_fetch(plan.handle, _ptr(res), _ptr(labels), _ptr(best), _stream(stream)))
    return res, labels, best


def ffe_plan_fetch_grid(plan, n, stream=None, want_err=False):
    """Omega(Delta) grids [n_q, n_pts, n] of a grid phase-scan plan (and their error bounds)."""
    om = np.zeros((plan.n_q, plan.n_pts, n))
    eb = np.zeros_like(om) if want_err else None
    _check(plan.ctx, lib().ffe_plan_fetch_grid(plan.handle, _ptr(om), _ptr(eb), _stream(stream)))
    return (om, eb) if want_err else om


def ffe_plan_stats(plan) -> dict:
    info = ffe_plan_info()
    _check(plan.ctx, lib().ffe_plan_stats(plan.handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in ffe_plan_info._fields_ if name != "reserved"}


def ffe_plan_kernel_ms(plan):
    ms = ctypes.c_double()
    n = ctypes.c_int32()
    _check(plan.ctx, lib().ffe_plan_kernel_ms(plan.handle, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def ffe_plan_destroy(plan):
    if plan.handle:
        lib().ffe_plan_destroy(plan.handle)
        plan.handle = None


def ffe_plan_minimize(ctx, params: np.ndarray, search=FFE_SEARCH_GRID, stream=None):
    ps = np.ascontiguousarray(params, dtype=PARAM_DTYPE)
    plan = _VP()
    _check(ctx, lib().ffe_plan_minimize(ctx, search, _ptr(ps), len(ps), _stream(stream), ctypes.byref(plan)))
    p = Plan(ctx, plan, 0, 0)
    p.n_params = len(ps)
    p.n_grid = int(ps["n"].sum()) if search == FFE_SEARCH_GRID else 0
    return p


def ffe_plan_fetch_minimize(plan, want_grid=False, stream=None):
    res = np.zeros(plan.n_params, dtype=RESULT_DTYPE)
    grid = np.zeros(plan.n_grid) if want_grid else None
    err = np.zeros(plan.n_grid) if want_grid else None
    _check(plan.ctx, lib().ffe_plan_fetch_minimize(plan.handle, _ptr(res), _ptr(grid), _ptr(err), _stream(stream)))
    return (res, grid, err) if want_grid else res


def ffe_plan_autotune(plan, stream=None) -> dict:
    kpt, block, target = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(plan.ctx, lib().ffe_plan_autotune(plan.handle, _stream(stream), ctypes.byref(kpt), ctypes.byref(block),
                                             ctypes.byref(target)))
    return {"kpt": kpt.value, "block": block.value, "item_target": target.value}


class Plan:
    def __init__(self, ctx, handle, n_q, n_pts):
        self.ctx, self.handle, self.n_q, self.n_pts = ctx, handle, n_q, n_pts

    def execute(self, stream=None):
        ffe_plan_execute(self, stream)

    def fetch(self, stream=None, labels=True):
        return ffe_plan_fetch(self, stream, labels)

    def fetch_minimize(self, want_grid=False, stream=None):
        return ffe_plan_fetch_minimize(self, want_grid, stream)

    def autotune(self, stream=None):
        return ffe_plan_autotune(self, stream)

    def stats(self):
        return ffe_plan_stats(self)

    def fetch_grid(self, n, stream=None, want_err=False):
        return ffe_plan_fetch_grid(self, n, stream, want_err)

    def kernel_ms(self):
        return ffe_plan_kernel_ms(self)

    def destroy(self):
        ffe_plan_destroy(self)


class Context:
    """Owning wrapper: ffe_create on construction, ffe_destroy on close()."""

    def __init__(self, prec=FFE_FP32C, U=2.0, eta_amp=1.0, model="raghu2", U_band=None, **params):
        self.nbands = MODELS[model][1]
        self.handle = ffe_create(prec=prec, U=U, eta_amp=eta_amp, model=model, U_band=U_band, **params)

    def omega(self, points, stream=None, bands=False):
        return ffe_omega(self.handle, points, stream, self.nbands if bands else 0)

    def minimize(self, params, search=FFE_SEARCH_GRID, want_grid=False, stream=None):
        return ffe_minimize(self.handle, params, search, want_grid, stream)

    def pair_susceptibility(self, N, qx, qy, h, T, stream=None):
        return ffe_pair_susceptibility(self.handle, N, qx, qy, h, T, self.nbands, stream)

    def minimize_bands(self, params, search=FFE_SEARCH_GRID, stream=None):
        return ffe_minimize_bands(self.handle, params, search, stream, self.nbands)

    def phase_scan(self, *a, **k):
        return ffe_phase_scan(self.handle, *a, **k)

    def plan_phase_scan(self, *a, **k):
        return ffe_plan_phase_scan(self.handle, *a, **k)

    def plan_minimize(self, params, search=FFE_SEARCH_GRID, stream=None):
        return ffe_plan_minimize(self.handle, params, search, stream)

    def close(self):
        if self.handle:
            ffe_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def points(N, qx, qy, h, T, delta) -> np.ndarray:
    """Pack broadcastable columns into an ffe_point array."""
    cols = np.broadcast_arrays(np.asarray(N), np.asarray(qx, float), np.asarray(qy, float),
                               np.asarray(h, float), np.asarray(T, float), np.asarray(delta, float))
    a = np.zeros(cols[0].size, dtype=POINT_DTYPE)
    for name, c in zip(("N", "qx", "qy", "h", "T", "delta"), cols):
        a[name] = c.ravel()
    return a


def params(N, qx, qy, h, T, lo, hi, n) -> np.ndarray:
    cols = np.broadcast_arrays(np.asarray(N), np.asarray(qx, float), np.asarray(qy, float),
                               np.asarray(h, float), np.asarray(T, float), np.asarray(lo, float),
                               np.asarray(hi, float), np.asarray(n))
    a = np.zeros(cols[0].size, dtype=PARAM_DTYPE)
    for name, c in zip(("N", "qx", "qy", "h", "T", "lo", "hi", "n"), cols):
        a[name] = c.ravel()
    return a
