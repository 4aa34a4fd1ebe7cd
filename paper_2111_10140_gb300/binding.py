"""ctypes binding of libanova_gb300.so (argument marshalling only).

Every function mirrors the C entry point of the same name declared in
``include/anova_gb300.h``; tensors are passed as raw device pointers together
with torch's current CUDA stream.  There is no fallback: if the library has not
been built (``__graft_entry__.build()``) or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ERANGE, ETIMEOUT, EBUSY = range(8)
FP64, FP32, MIXED = 1, 2, 3

_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pf64 = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "anova_fastsum_plan": (_i32, [_vp, _i64, _i32, _i64, _pi32, _i32, _pf64, _f64, _pi32, _i32, _f64,
                                  _f64, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "anova_matvec": (_i32, [_vp, _i32, _vp, _vp, _i32, _i64, _vp]),
    "krr_cg_solve": (_i32, [_vp, _f64, _vp, _vp, _i32, _i64, _f64, _i32, _pi32, _pf64, _vp]),
    "krr_predict": (_i32, [_vp, _vp, _vp, _i64, _i64, _vp, _vp]),
    "krr_predict_noalloc": (_i32, [_vp, _vp, _vp, _i64, _i64, _vp, _vp]),
    "anova_direct_matvec": (_i32, [_vp, _i64, _i64, _vp, _i64, _i64, _i32, _pi32, _i32, _pf64, _f64, _i32, _vp,
                                   _vp, _vp]),
    "anova_plan_set_graphs": (_i32, [_vp, _i32]),
    "anova_plan_set_tensor_cores": (_i32, [_vp, _i32]),
    "anova_plan_set_overlap": (_i32, [_vp, _i32]),
    "anova_autotune_kernels": (_i32, [_vp, _i32, _pi32, _pf64, _vp]),
    "anova_plan_set_kernels": (_i32, [_vp, _pi32]),
    "anova_plan_get_kernels": (_i32, [_vp, _pi32]),
    "anova_fastsum_plan_bins": (_i32, [_vp, _i64, _i32, _i64, _pi32, _i32, _pf64, _f64, _pi32, _i32, _f64, _f64,
                                       _i32, _i32, _pi32, _vp, ctypes.POINTER(_vp)]),
    "anova_autotune_bins": (_i32, [_vp, _i64, _i32, _i64, _pi32, _i32, _pf64, _f64, _pi32, _i32, _f64, _f64,
                                   _i32, _i32, _i32, _pi32, _pf64, _vp]),
    "anova_plan_window_bins": (_i32, [_vp, _i32, _pi32, _pi32, _pi32]),
    "anova_plan_bin_rule": (_i32, [_i32, _i32, _i32, _f64, _pi32, _pi32, _pi32, _pi32, _pi32]),
    "anova_wait_timeouts": (_i64, []),
    "anova_debug_wait_probe": (_i32, [_i32, _vp]),
    "anova_zscore_fit": (_i32, [_vp, _i64, _i32, _i64, _vp, _vp, _vp]),
    "anova_zscore_apply": (_i32, [_vp, _i64, _i32, _i64, _vp, _vp, _vp]),
    "anova_mis": (_i32, [_vp, _i64, _i32, _i64, _vp, _i32, _i32, _pf64, _vp]),
    "anova_mis_fine_bins": (_i32, [_vp, _i64, _i32, _i64, _vp, _vp]),
    "anova_windows_from_mis": (_i32, [_pf64, _i32, _f64, _pi32, _pi32]),
    "anova_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "anova_batch_layout": (_i32, [_vp, _pi64]),
    "anova_batch_matvec": (_i32, [_vp, _vp, _vp, _vp]),
    "krr_batch_cg_solve": (_i32, [_vp, _pf64, _vp, _vp, _f64, _i32, _pi32, _pf64, _vp]),
    "krr_batch_cg_solve_refined": (_i32, [_vp, _pf64, _vp, _vp, _f64, _i32, _pi32, _pf64, _vp]),
    "anova_batch_destroy": (None, [_vp]),
    "krr_model_create": (_i32, [_vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "krr_model_predict": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp]),
    "krr_model_destroy": (None, [_vp]),
    "anova_server_create": (_i32, [_i32, _i64, ctypes.POINTER(_vp)]),
    "anova_server_submit_fit": (_i32, [_vp, _vp, _i64, _i32, _pi32, _i32, _f64, _pi32, _i32, _f64, _f64, _vp,
                                       _f64, _i32, _pi64]),
    "anova_server_submit_predict": (_i32, [_vp, _i64, _vp, _i64, _vp, _pi64]),
    "anova_server_wait": (_i32, [_vp, _i64, _pi32, _pf64, _pi32, _pf64]),
    "anova_server_release": (_i32, [_vp, _i64]),
    "anova_server_stats": (_i32, [_vp, _pf64, _pf64, _pi64, _pi64]),
    "anova_server_destroy": (None, [_vp]),
    "anova_plan_destroy": (None, [_vp]),
    "anova_status_string": (ctypes.c_char_p, [_i32]),
    "anova_last_error": (ctypes.c_char_p, []),
    "anova_plan_window": (_i32, [_vp, _i32, _pf64, _pf64, _pf64, _pi32, _pi32, _pi32]),
    "anova_debug_spread": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "anova_debug_diag": (_i32, [_vp, _i32, _pf64]),
    "anova_set_profiling": (_i32, [_vp, _i32]),
    "anova_stage_times": (_i32, [_vp, _pf64, _pi64, _i32]),
    "krr_model_alpha": (_i32, [_vp, _vp, _vp]),
    "anova_debug_fail_alloc": (_i32, [_i64]),
    "anova_debug_memory": (_i32, [_pi64, _pi64, _pi64]),
    "anova_server_fit_alpha": (_i32, [_vp, _i64, _vp, _vp]),
    "anova_server_set_fit_wait_bound": (_i32, [_vp, _f64]),
    "anova_plan_dense3_kernels": (_i32, [_vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_char_p)]),
}


class AnovaError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = lib().anova_last_error().decode()
        super().__init__(f"{where}: {lib().anova_status_string(status).decode()} ({detail})")


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status, where, allow=(OK,)):
    if status not in allow:
        raise AnovaError(status, where)
    return status


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _require_cuda(t, name, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def windows_array(windows) -> np.ndarray:
    out = -np.ones((len(windows), 3), dtype=np.int32)
    for l, w in enumerate(windows):
        out[l, :len(w)] = w
    return out


class Plan:
    """Owning handle of an anova_plan (destroyed with the object)."""

    def __init__(self, handle, N, d, P, precision):
        self.handle = handle
        self.N, self.d, self.P, self.precision = N, d, P, precision

    def close(self):
        if self.handle:
            lib().anova_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def anova_fastsum_plan(points, windows, ell, n=None, m=6, sigma=2.0, eps_B=1.0 / 16, p=8,
                       precision=FP64, weights=None, stream=None) -> Plan:
    import torch
    _require_cuda(points, "points", torch.float64)
    N, d = points.shape
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else np.ascontiguousarray(windows, np.int32)
    P = W.shape[0]
    wts = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    nv = None if n is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n, np.int32), (P,)), dtype=np.int32)
    h = ctypes.c_void_p()
    st = lib().anova_fastsum_plan(
        _ptr(points), N, d, d, W.ctypes.data_as(_pi32), P,
        wts.ctypes.data_as(_pf64) if wts is not None else None, float(ell),
        nv.ctypes.data_as(_pi32) if nv is not None else None, int(m), float(sigma), float(eps_B), int(p),
        int(precision), _stream(stream), ctypes.byref(h))
    _check(st, "anova_fastsum_plan")
    return Plan(h, N, d, P, precision)


def _plan_args(points, windows, n):
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else np.ascontiguousarray(windows, np.int32)
    P = W.shape[0]
    nv = None if n is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n, np.int32), (P,)), dtype=np.int32)
    return W, P, nv


def anova_fastsum_plan_bins(points, windows, ell, bin_side, n=None, m=6, sigma=2.0, eps_B=1.0 / 16, p=8,
                            precision=FP64, weights=None, stream=None) -> Plan:
    import torch
    _require_cuda(points, "points", torch.float64)
    N, d = points.shape
    W, P, nv = _plan_args(points, windows, n)
    wts = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    bs = np.ascontiguousarray(bin_side, dtype=np.int32)
    h = ctypes.c_void_p()
    st = lib().anova_fastsum_plan_bins(
        _ptr(points), N, d, d, W.ctypes.data_as(_pi32), P, wts.ctypes.data_as(_pf64) if wts is not None else None,
        float(ell), nv.ctypes.data_as(_pi32) if nv is not None else None, int(m), float(sigma), float(eps_B), int(p),
        int(precision), bs.ctypes.data_as(_pi32), _stream(stream), ctypes.byref(h))
    _check(st, "anova_fastsum_plan_bins")
    return Plan(h, N, d, P, precision)


def anova_autotune_bins(points, windows, ell, n=None, m=6, sigma=2.0, eps_B=1.0 / 16, p=8, precision=FP32,
                        reps=10, stream=None):
    """Returns (bin_side [3], ms per product)."""
    import torch
    _require_cuda(points, "points", torch.float64)
    N, d = points.shape
    W, P, nv = _plan_args(points, windows, n)
    bs = np.zeros(3, dtype=np.int32)
    ms = ctypes.c_double()
    st = lib().anova_autotune_bins(_ptr(points), N, d, d, W.ctypes.data_as(_pi32), P, None, float(ell),
                                   nv.ctypes.data_as(_pi32) if nv is not None else None, int(m), float(sigma),
                                   float(eps_B), int(p), int(precision), int(reps), bs.ctypes.data_as(_pi32),
                                   ctypes.byref(ms), _stream(stream))
    _check(st, "anova_autotune_bins")
    return [int(v) for v in bs], ms.value


SPREAD3_FORMS = ("fma", "mma.sync", "mma.sync pipelined", "mma.sync fp16 split")
GATHER3_FORMS = ("fma", "mma.sync", "tcgen05", "tcgen05 persistent")


def anova_autotune_kernels(plan: Plan, reps=10, stream=None):
    """Sets the plan's fastest kernel forms; returns ({"spread3", "gather3", "schedule"}, ms per product)."""
    c = np.zeros(3, dtype=np.int32)
    ms = ctypes.c_double()
    _check(lib().anova_autotune_kernels(plan.handle, int(reps), c.ctypes.data_as(_pi32), ctypes.byref(ms),
                                        _stream(stream)), "anova_autotune_kernels")
    return {"spread3": SPREAD3_FORMS[c[0]], "gather3": GATHER3_FORMS[c[1]], "schedule": int(c[2])}, ms.value


def anova_plan_set_kernels(plan: Plan, spread3, gather3, schedule):
    """Kernel forms by name (SPREAD3_FORMS, GATHER3_FORMS) and the 1-D / 2-D schedule (0..3)."""
    c = np.array([SPREAD3_FORMS.index(spread3), GATHER3_FORMS.index(gather3), int(schedule)], dtype=np.int32)
    _check(lib().anova_plan_set_kernels(plan.handle, c.ctypes.data_as(_pi32)), "anova_plan_set_kernels")


def anova_plan_get_kernels(plan: Plan) -> dict:
    c = np.zeros(3, dtype=np.int32)
    _check(lib().anova_plan_get_kernels(plan.handle, c.ctypes.data_as(_pi32)), "anova_plan_get_kernels")
    return {"spread3": SPREAD3_FORMS[c[0]], "gather3": GATHER3_FORMS[c[1]], "schedule": int(c[2])}


def anova_plan_window_bins(plan: Plan, l: int) -> dict:
    t, r, dn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().anova_plan_window_bins(plan.handle, l, ctypes.byref(t), ctypes.byref(r), ctypes.byref(dn)),
           "anova_plan_window_bins")
    return {"bin_side": t.value, "region": r.value, "dense": bool(dn.value)}


def anova_matvec(plan: Plan, alpha, out, stream=None):
    import torch
    _require_cuda(alpha, "alpha")
    _require_cuda(out, "out", alpha.dtype)
    dtype = FP64 if alpha.dtype == torch.float64 else FP32 if alpha.dtype == torch.float32 else None
    if dtype is None:
        raise ValueError("alpha must be float64 or float32")
    nrhs = 1 if alpha.dim() == 1 else alpha.shape[0]
    ld = alpha.shape[-1]
    _check(lib().anova_matvec(plan.handle, dtype, _ptr(alpha), _ptr(out), nrhs, ld, _stream(stream)),
           "anova_matvec")
    return out


def krr_cg_solve(plan: Plan, lam, y, alpha, tol, maxit, stream=None):
    """Returns (status, iterations per column, true relative residual per column)."""
    import torch
    _require_cuda(y, "y", torch.float64)
    _require_cuda(alpha, "alpha", torch.float64)
    nrhs = 1 if y.dim() == 1 else y.shape[0]
    ld = y.shape[-1]
    its = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs, dtype=np.float64)
    st = lib().krr_cg_solve(plan.handle, float(lam), _ptr(y), _ptr(alpha), nrhs, ld, float(tol), int(maxit),
                            its.ctypes.data_as(_pi32), rel.ctypes.data_as(_pf64), _stream(stream))
    _check(st, "krr_cg_solve", allow=(OK, ENOCONV))
    return st, its, rel


def krr_predict(plan: Plan, alpha, Z, out, stream=None):
    import torch
    _require_cuda(alpha, "alpha", torch.float64)
    _require_cuda(Z, "Z", torch.float64)
    _require_cuda(out, "out", torch.float64)
    M = Z.shape[0]
    _check(lib().krr_predict(plan.handle, _ptr(alpha), _ptr(Z), M, Z.shape[1], _ptr(out), _stream(stream)),
           "krr_predict")
    return out


def krr_predict_noalloc(plan: Plan, alpha, Z, out, stream=None):
    """krr_predict without device allocation inside the call (see the header)."""
    import torch
    _require_cuda(alpha, "alpha", torch.float64)
    _require_cuda(Z, "Z", torch.float64)
    _require_cuda(out, "out", torch.float64)
    _check(lib().krr_predict_noalloc(plan.handle, _ptr(alpha), _ptr(Z), Z.shape[0], Z.shape[1], _ptr(out),
                                     _stream(stream)), "krr_predict_noalloc")
    return out


def anova_direct_matvec(Z, X, windows, ell, alpha, out, weights=None, dtype=FP64, stream=None):
    """Exact kernel sum out = sum_l eta_l sum_j alpha_j kappa_l(z_i, x_j) on the GPU."""
    import torch
    for t, nm in ((Z, "Z"), (X, "X"), (alpha, "alpha"), (out, "out")):
        _require_cuda(t, nm, torch.float64)
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else np.ascontiguousarray(windows, np.int32)
    wts = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    _check(lib().anova_direct_matvec(_ptr(Z), Z.shape[0], Z.shape[1], _ptr(X), X.shape[0], X.shape[1], X.shape[1],
                                     W.ctypes.data_as(_pi32), W.shape[0],
                                     wts.ctypes.data_as(_pf64) if wts is not None else None, float(ell),
                                     int(dtype), _ptr(alpha), _ptr(out), _stream(stream)), "anova_direct_matvec")
    return out


def anova_plan_window(plan: Plan, l: int) -> dict:
    c = (ctypes.c_double * 3)()
    s, e = ctypes.c_double(), ctypes.c_double()
    dims, n, nos = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().anova_plan_window(plan.handle, l, c, ctypes.byref(s), ctypes.byref(e), ctypes.byref(dims),
                                   ctypes.byref(n), ctypes.byref(nos)), "anova_plan_window")
    return {"centre": np.array(c[:dims.value]), "scale": s.value, "ell_l": e.value, "dims": dims.value,
            "n": n.value, "nos": nos.value}


def anova_debug_spread(plan: Plan, l: int, alpha, grid, stream=None):
    import torch
    dtype = FP64 if alpha.dtype == torch.float64 else FP32
    _check(lib().anova_debug_spread(plan.handle, l, dtype, _ptr(alpha), _ptr(grid), _stream(stream)),
           "anova_debug_spread")
    return grid


def anova_debug_diag(plan: Plan, l: int) -> np.ndarray:
    info = anova_plan_window(plan, l)
    D = np.zeros(info["n"] ** info["dims"])
    _check(lib().anova_debug_diag(plan.handle, l, D.ctypes.data_as(_pf64)), "anova_debug_diag")
    return D.reshape((info["n"],) * info["dims"])


def anova_set_profiling(plan: Plan, enable: bool):
    _check(lib().anova_set_profiling(plan.handle, int(bool(enable))), "anova_set_profiling")


def anova_plan_set_graphs(plan: Plan, enable: bool):
    _check(lib().anova_plan_set_graphs(plan.handle, 1 if enable else 0), "anova_plan_set_graphs")


def anova_plan_set_tensor_cores(plan: Plan, enable):
    """enable: False (FMA kernels), True (the default kernels) or 2 (also the tcgen05 3-D spread)."""
    mode = 2 if enable == 2 else (1 if enable else 0)
    _check(lib().anova_plan_set_tensor_cores(plan.handle, mode), "anova_plan_set_tensor_cores")


def anova_plan_set_overlap(plan: Plan, mode: int):
    _check(lib().anova_plan_set_overlap(plan.handle, int(mode)), "anova_plan_set_overlap")


def anova_stage_times(plan: Plan):
    ms = (ctypes.c_double * 8)()
    la = (ctypes.c_int64 * 8)()
    k = lib().anova_stage_times(plan.handle, ms, la, 8)
    return list(ms[:k]), list(la[:k])


def anova_debug_fail_alloc(k: int):
    """Make the k-th device allocation of the library from now on fail (0: off)."""
    _check(lib().anova_debug_fail_alloc(int(k)), "anova_debug_fail_alloc")


def anova_debug_memory() -> dict:
    """Free device bytes and the default stream-ordered pool's used / reserved bytes."""
    f, u, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().anova_debug_memory(ctypes.byref(f), ctypes.byref(u), ctypes.byref(r)), "anova_debug_memory")
    return {"free": f.value, "pool_used": u.value, "pool_reserved": r.value}


def anova_dense3_kernels(plan: Plan) -> dict:
    """Kernel names of the plan's FP32 3-D spread and gather ("<R>": the region size)."""
    sp, ga = ctypes.c_char_p(), ctypes.c_char_p()
    _check(lib().anova_plan_dense3_kernels(plan.handle, ctypes.byref(sp), ctypes.byref(ga)),
           "anova_plan_dense3_kernels")
    return {"spread": sp.value.decode(), "gather": ga.value.decode()}


def anova_zscore_fit(X, stream=None):
    """(mean, sd) device tensors of the columns of X (device, N x d float64)."""
    import torch
    _require_cuda(X, "X", torch.float64)
    mean = torch.empty(X.shape[1], dtype=torch.float64, device=X.device)
    sd = torch.empty_like(mean)
    _check(lib().anova_zscore_fit(_ptr(X), X.shape[0], X.shape[1], X.stride(0), _ptr(mean), _ptr(sd),
                                  _stream(stream)), "anova_zscore_fit")
    return mean, sd


def anova_zscore_apply(X, mean, sd, stream=None):
    import torch
    _require_cuda(X, "X", torch.float64)
    _check(lib().anova_zscore_apply(_ptr(X), X.shape[0], X.shape[1], X.stride(0), _ptr(mean), _ptr(sd),
                                    _stream(stream)), "anova_zscore_apply")
    return X


def anova_mis(X, labels, nclass, bins=16, stream=None):
    import torch
    _require_cuda(X, "X", torch.float64)
    _require_cuda(labels, "labels", torch.int32)
    out = np.zeros(X.shape[1], dtype=np.float64)
    _check(lib().anova_mis(_ptr(X), X.shape[0], X.shape[1], X.stride(0), _ptr(labels), int(nclass), int(bins),
                           out.ctypes.data_as(_pf64), _stream(stream)), "anova_mis")
    return out


def anova_mis_fine_bins(X, stream=None):
    """Fine bin (0..4095) of every element of X, the integer intermediate of anova_mis."""
    import torch
    _require_cuda(X, "X", torch.float64)
    out = torch.empty(X.shape, dtype=torch.int32, device=X.device)
    _check(lib().anova_mis_fine_bins(_ptr(X), X.shape[0], X.shape[1], X.stride(0), _ptr(out), _stream(stream)),
           "anova_mis_fine_bins")
    return out


def anova_windows_from_mis(scores, threshold=0.0):
    s = np.ascontiguousarray(scores, dtype=np.float64)
    w = np.full(3 * len(s), -1, dtype=np.int32)
    P = ctypes.c_int32()
    _check(lib().anova_windows_from_mis(s.ctypes.data_as(_pf64), len(s), float(threshold), w.ctypes.data_as(_pi32),
                                        ctypes.byref(P)), "anova_windows_from_mis")
    return [tuple(int(f) for f in w[3 * p:3 * p + 3] if f >= 0) for p in range(P.value)]


def anova_plan_bin_rule(dims, n, m, sigma=2.0, bin_side=None):
    """Binning a plan would give one window (no GPU): side, region, dense, nbins."""
    req = None
    if bin_side is not None:
        req = np.ascontiguousarray(bin_side, dtype=np.int32)
        assert req.shape == (3,)
    out = [ctypes.c_int32() for _ in range(4)]
    _check(lib().anova_plan_bin_rule(int(dims), int(n), int(m), float(sigma),
                                     req.ctypes.data_as(_pi32) if req is not None else None,
                                     *[ctypes.byref(o) for o in out]), "anova_plan_bin_rule")
    return {"bin_side": out[0].value, "region": out[1].value, "dense": bool(out[2].value), "nbins": out[3].value}


def anova_wait_timeouts():
    return int(lib().anova_wait_timeouts())


def anova_debug_wait_probe(polls, stream=None):
    """Status of the bounded-wait probe (ETIMEOUT when its wait gave up)."""
    return int(lib().anova_debug_wait_probe(int(polls), _stream(stream)))


class Batch:
    """anova_batch over plans (kept alive here) with nrhs right-hand sides each."""

    def __init__(self, plans, nrhs, stream=None):
        arr = (_vp * len(plans))(*[p.handle.value for p in plans])
        h = ctypes.c_void_p()
        _check(lib().anova_batch_create(arr, len(plans), int(nrhs), _stream(stream), ctypes.byref(h)),
               "anova_batch_create")
        self.handle = h
        self.plans = list(plans)
        self.nrhs = int(nrhs)
        off = np.zeros(len(plans) + 1, dtype=np.int64)
        _check(lib().anova_batch_layout(h, off.ctypes.data_as(_pi64)), "anova_batch_layout")
        self.offsets = off

    @property
    def size(self):
        return int(self.offsets[-1])

    def block(self, flat, p):
        """View of problem p's nrhs x N_p block of a flat vector."""
        return flat[self.offsets[p]:self.offsets[p + 1]].view(self.nrhs, -1)

    def matvec(self, x, y, stream=None):
        import torch
        _require_cuda(x, "x", torch.float64)
        _require_cuda(y, "y", torch.float64)
        _check(lib().anova_batch_matvec(self.handle, _ptr(x), _ptr(y), _stream(stream)), "anova_batch_matvec")
        return y

    def cg_solve(self, lambdas, y, alpha, tol, maxit, stream=None, refined=False):
        """Returns (status, iterations, relres), both arrays of problems x nrhs.
        refined=True: krr_batch_cg_solve_refined (FP64 residual)."""
        import torch
        _require_cuda(y, "y", torch.float64)
        _require_cuda(alpha, "alpha", torch.float64)
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambdas, np.float64), (len(self.plans),)))
        ns = len(self.plans) * self.nrhs
        its = np.zeros(ns, dtype=np.int32)
        rr = np.zeros(ns, dtype=np.float64)
        fn = lib().krr_batch_cg_solve_refined if refined else lib().krr_batch_cg_solve
        st = fn(self.handle, lam.ctypes.data_as(_pf64), _ptr(y), _ptr(alpha), float(tol), int(maxit),
                its.ctypes.data_as(_pi32), rr.ctypes.data_as(_pf64), _stream(stream))
        _check(st, "krr_batch_cg_solve", allow=(OK, ENOCONV))
        return st, its.reshape(len(self.plans), self.nrhs), rr.reshape(len(self.plans), self.nrhs)

    def close(self):
        if self.handle:
            lib().anova_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """A fitted model (krr_model_create): the plan must outlive it."""

    def __init__(self, plan: Plan, alpha, stream=None):
        import torch
        _require_cuda(alpha, "alpha", torch.float64)
        h = ctypes.c_void_p()
        _check(lib().krr_model_create(plan.handle, _ptr(alpha), _stream(stream), ctypes.byref(h)),
               "krr_model_create")
        self.handle = h
        self.plan = plan

    def predict(self, Z, out, stream=None):
        import torch
        _require_cuda(Z, "Z", torch.float64)
        _require_cuda(out, "out", torch.float64)
        _check(lib().krr_model_predict(self.handle, _ptr(Z), Z.shape[0], Z.shape[1], _ptr(out), _stream(stream)),
               "krr_model_predict")
        return out

    def alpha(self, out, stream=None):
        """Copy the model's coefficients into `out` (device, float64, N)."""
        import torch
        _require_cuda(out, "out", torch.float64)
        _check(lib().krr_model_alpha(self.handle, _ptr(out), _stream(stream)), "krr_model_alpha")
        return out

    def close(self):
        if self.handle:
            lib().krr_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Handle of an anova_server (see the header); tensors passed in must stay
    alive until the corresponding wait() has returned."""

    def __init__(self, n_workers=4, hbm_budget_bytes=150 << 30):
        h = ctypes.c_void_p()
        _check(lib().anova_server_create(int(n_workers), int(hbm_budget_bytes), ctypes.byref(h)),
               "anova_server_create")
        self.handle = h
        self._keep = {}

    def submit_fit(self, points, windows, ell, y, lam, n=None, m=6, eps_B=1.0 / 16, tol=1e-6, maxit=5000):
        import torch
        _require_cuda(points, "points", torch.float64)
        _require_cuda(y, "y", torch.float64)
        W = windows_array(windows)
        P = W.shape[0]
        nv = None if n is None else np.ascontiguousarray(np.broadcast_to(np.asarray(n, np.int32), (P,)), np.int32)
        t = ctypes.c_int64()
        _check(lib().anova_server_submit_fit(self.handle, _ptr(points), points.shape[0], points.shape[1],
                                             W.ctypes.data_as(_pi32), P, float(ell),
                                             nv.ctypes.data_as(_pi32) if nv is not None else None, int(m),
                                             float(eps_B), float(lam), _ptr(y), float(tol), int(maxit),
                                             ctypes.byref(t)), "anova_server_submit_fit")
        self._keep[t.value] = (points, y)
        return t.value

    def submit_predict(self, model, Z, out):
        import torch
        _require_cuda(Z, "Z", torch.float64)
        _require_cuda(out, "out", torch.float64)
        t = ctypes.c_int64()
        _check(lib().anova_server_submit_predict(self.handle, int(model), _ptr(Z), Z.shape[0], _ptr(out),
                                                 ctypes.byref(t)), "anova_server_submit_predict")
        self._keep[t.value] = (Z, out)
        return t.value

    def wait(self, ticket):
        st, lat, it, rr = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().anova_server_wait(self.handle, int(ticket), ctypes.byref(st), ctypes.byref(lat),
                                       ctypes.byref(it), ctypes.byref(rr)), "anova_server_wait")
        self._keep.pop(ticket, None)
        return {"status": st.value, "latency_ms": lat.value, "iterations": it.value, "relres": rr.value}

    def release(self, model):
        _check(lib().anova_server_release(self.handle, int(model)), "anova_server_release")

    def fit_alpha(self, fit, out, stream=None):
        """Copy a served fit's coefficients into `out` (device, float64, N)."""
        import torch
        _require_cuda(out, "out", torch.float64)
        _check(lib().anova_server_fit_alpha(self.handle, int(fit), _ptr(out), _stream(stream)),
               "anova_server_fit_alpha")
        return out

    def set_fit_wait_bound(self, max_wait_ms):
        """Refuse fits (EBUSY at submission) whose expected queue wait exceeds max_wait_ms (0: never)."""
        _check(lib().anova_server_set_fit_wait_bound(self.handle, float(max_wait_ms)),
               "anova_server_set_fit_wait_bound")

    def stats(self):
        p50, p99 = ctypes.c_double(), ctypes.c_double()
        n, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().anova_server_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n),
                                        ctypes.byref(b)), "anova_server_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "completed": n.value, "bytes_in_use": b.value}

    def close(self):
        if self.handle:
            lib().anova_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
