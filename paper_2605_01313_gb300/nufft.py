"""Python binding of the dfsnufft C ABI (include/dfsnufft.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The low-level functions keep the C names; :class:`Plan` wraps them
for torch tensors (device memory and the current CUDA stream come from torch).
The library must have been built (``python -m paper_2605_01313_gb300.build``);
there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

F64 = 0
F32 = 1

OK = 0
ERR_INVALID_ARG = 1
ERR_TOL_UNATTAINABLE = 2
ERR_NO_POINTS = 3
ERR_OOM = 4
ERR_CUDA = 5
ERR_UNSUPPORTED = 6
ERR_TIMEOUT = 7

# Every symbol include/dfsnufft.h declares.
EXPORTS = (
    "dfsnufft_plan_create", "dfsnufft_set_points", "dfsnufft_execute",
    "dfsnufft_set_points_host", "dfsnufft_execute_host", "dfsnufft_execute_points_host",
    "dfsnufft_destroy",
    "dfsnufft_strerror", "dfsnufft_plan_last_error", "dfsnufft_plan_get_params",
    "dfsnufft_choose_params", "dfsnufft_es_kernel", "dfsnufft_kernel_ft", "dfsnufft_version",
    "dfsnufft_plan_enable_timing", "dfsnufft_plan_read_timing", "dfsnufft_plan_point_stats",
    "dfsnufft_probe_fma_rate", "dfsnufft_execute_noalloc", "dfsnufft_plan_check",
    "dfsnufft_es_horner", "dfsnufft_plan_create_batch", "dfsnufft_set_points_batch",
    "dfsnufft_ensemble_create", "dfsnufft_ensemble_run", "dfsnufft_ensemble_check",
    "dfsnufft_ensemble_plan", "dfsnufft_ensemble_destroy",
    "dfsnufft_server_create", "dfsnufft_server_submit", "dfsnufft_server_wait",
    "dfsnufft_server_stats_get", "dfsnufft_server_destroy",
    "dfsnufft_choose_params_opts", "dfsnufft_plan_create_opts", "dfsnufft_ensemble_create_opts",
    "dfsnufft_server_create_opts", "dfsnufft_autotune", "dfsnufft_selftest_wait_timeout",
    "dfsnufft_execute_pr", "dfsnufft_grid_to_coeffs", "dfsnufft_interpolate_grid",
    "dfsnufft_departure_points", "dfsnufft_rotate_to_arrival", "dfsnufft_lagrange_interp",
    "dfsnufft_plan_latitudes", "dfsnufft_plan_host_copy_bytes",
    "dfsnufft_ensemble_set_persistent", "dfsnufft_ensemble_selftest_queue_timeout",
)
REAL_FIELDS = 1
KEEP_ORDER = 2
GAUSS_GRID = 4
N_STAGES = 4
STAGES = ("set_points", "theta_pass", "phi_pass", "interp")


class Params(ctypes.Structure):
    _fields_ = [("n_lon", ctypes.c_int), ("n_lat", ctypes.c_int), ("N1", ctypes.c_int),
                ("N2", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("w", ctypes.c_int), ("beta", ctypes.c_double), ("tol", ctypes.c_double),
                ("dtype", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("sigma", ctypes.c_int), ("flags", ctypes.c_uint)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Options(ctypes.Structure):
    """dfsnufft_options: zero fields take the defaults."""
    _fields_ = [("flags", ctypes.c_uint), ("sigma", ctypes.c_int), ("w", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int)]

    @classmethod
    def make(cls, real_fields=False, sigma=0, w=0, tile=None, keep_order=False, gauss=False):
        o = cls()
        o.flags = ((REAL_FIELDS if real_fields else 0) | (KEEP_ORDER if keep_order else 0)
                   | (GAUSS_GRID if gauss else 0))
        o.sigma = int(sigma or 0)
        o.w = int(w or 0)
        if tile:
            o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        return o

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneArgs(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_int), ("n_lon", ctypes.c_int), ("n_lat", ctypes.c_int),
                ("tol", ctypes.c_double), ("dtype", ctypes.c_int), ("n_fields", ctypes.c_int),
                ("flags", ctypes.c_uint), ("n_points", ctypes.c_void_p),
                ("lon", ctypes.c_void_p), ("colat", ctypes.c_void_p),
                ("coeffs", ctypes.c_void_p), ("steps", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("opts", Options), ("prm", Params), ("ms", ctypes.c_double),
                ("err", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {"opts": self.opts.as_dict(), "params": self.prm.as_dict(), "ms": self.ms,
                "err": self.err, "status": self.status}


class Request(ctypes.Structure):
    _fields_ = [("n_lon", ctypes.c_int), ("n_lat", ctypes.c_int), ("n_points", ctypes.c_int64),
                ("lon", ctypes.c_void_p), ("colat", ctypes.c_void_p), ("coeffs", ctypes.c_void_p),
                ("values", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("members", ctypes.c_int64), ("slots", ctypes.c_int),
                ("reserved_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DfsError(RuntimeError):
    def __init__(self, status, detail=""):
        self.status = status
        msg = "dfsnufft: %s (status %d)" % (_strerror(status), status)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("dfsnufft CUDA library missing at %s; build it with "
                               "`python -m paper_2605_01313_gb300.build`" % path)
        L = ctypes.CDLL(path)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.dfsnufft_plan_create.argtypes = [i32, i32, f64, i32, i32, vp, ctypes.POINTER(vp)]
        L.dfsnufft_plan_create_batch.argtypes = [i32, i32, i32, f64, i32, i32, vp,
                                                 ctypes.POINTER(vp)]
        L.dfsnufft_plan_create_opts.argtypes = [i32, i32, i32, f64, i32, i32,
                                                ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.dfsnufft_choose_params_opts.argtypes = [i32, i32, f64, i32, ctypes.POINTER(Options),
                                                  ctypes.POINTER(Params)]
        L.dfsnufft_ensemble_create_opts.argtypes = [i32, vp, vp, vp, f64, i32, i32,
                                                    ctypes.POINTER(Options), vp,
                                                    ctypes.POINTER(vp)]
        L.dfsnufft_set_points_batch.argtypes = [vp, vp, vp, vp]
        L.dfsnufft_ensemble_create.argtypes = [i32, vp, vp, vp, f64, i32, i32, vp,
                                               ctypes.POINTER(vp)]
        L.dfsnufft_ensemble_run.argtypes = [vp, vp, vp, vp, vp, vp]
        L.dfsnufft_ensemble_check.argtypes = [vp]
        L.dfsnufft_ensemble_plan.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.dfsnufft_ensemble_destroy.argtypes = [vp]
        L.dfsnufft_ensemble_set_persistent.argtypes = [vp, i32]
        L.dfsnufft_ensemble_selftest_queue_timeout.argtypes = [vp, ctypes.c_longlong]
        L.dfsnufft_server_create.argtypes = [f64, i32, i32, i64, i32, ctypes.POINTER(vp)]
        L.dfsnufft_autotune.argtypes = [ctypes.POINTER(TuneArgs), ctypes.POINTER(TuneResult), i32,
                                        ctypes.POINTER(i32), ctypes.POINTER(Options)]
        L.dfsnufft_server_create_opts.argtypes = [f64, i32, i32, i64, i32,
                                                  ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.dfsnufft_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(i64)]
        L.dfsnufft_server_wait.argtypes = [vp, i64, f64, ctypes.POINTER(i32), ctypes.POINTER(f64)]
        L.dfsnufft_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.dfsnufft_server_destroy.argtypes = [vp]
        L.dfsnufft_set_points.argtypes = [vp, i64, vp, vp]
        L.dfsnufft_set_points_host.argtypes = [vp, i64, vp, vp]
        L.dfsnufft_execute.argtypes = [vp, vp, vp]
        L.dfsnufft_execute_pr.argtypes = [vp, i32, i32, vp, vp]
        L.dfsnufft_grid_to_coeffs.argtypes = [vp, vp, vp, vp]
        L.dfsnufft_interpolate_grid.argtypes = [vp, vp, vp, vp]
        L.dfsnufft_execute_host.argtypes = [vp, vp, vp]
        L.dfsnufft_execute_points_host.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp]
        L.dfsnufft_destroy.argtypes = [vp]
        L.dfsnufft_strerror.argtypes = [i32]
        L.dfsnufft_strerror.restype = ctypes.c_char_p
        L.dfsnufft_plan_last_error.argtypes = [vp]
        L.dfsnufft_plan_last_error.restype = ctypes.c_char_p
        L.dfsnufft_plan_get_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.dfsnufft_plan_check.argtypes = [vp]
        L.dfsnufft_choose_params.argtypes = [i32, i32, f64, i32, ctypes.POINTER(Params)]
        L.dfsnufft_es_kernel.argtypes = [f64, i32, f64]
        L.dfsnufft_es_kernel.restype = f64
        L.dfsnufft_kernel_ft.argtypes = [i32, f64, i32, i32, vp]
        L.dfsnufft_es_horner.argtypes = [i32, f64, vp]
        L.dfsnufft_version.restype = ctypes.c_char_p
        L.dfsnufft_plan_enable_timing.argtypes = [vp, i32]
        L.dfsnufft_plan_read_timing.argtypes = [vp, vp, vp]
        L.dfsnufft_plan_point_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.dfsnufft_plan_host_copy_bytes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                                    ctypes.POINTER(i64)]
        L.dfsnufft_probe_fma_rate.argtypes = [i32, f64, ctypes.POINTER(f64)]
        L.dfsnufft_selftest_wait_timeout.argtypes = [ctypes.c_longlong, ctypes.POINTER(i32),
                                                     ctypes.POINTER(f64)]
        L.dfsnufft_execute_noalloc.argtypes = [i32, i32, f64, i32, i32, i64, vp, vp, vp, vp, vp]
        L.dfsnufft_departure_points.argtypes = [i32, i32, i32, i32, i32, f64, vp, vp, vp, vp, vp,
                                                vp]
        L.dfsnufft_rotate_to_arrival.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp, i64, vp,
                                                 vp, vp]
        L.dfsnufft_plan_latitudes.argtypes = [vp, vp]
        L.dfsnufft_lagrange_interp.argtypes = [i32, i32, i32, vp, i32, i32, i64, vp, vp, vp, vp,
                                               vp]
        for name in EXPORTS:
            if name not in ("dfsnufft_strerror", "dfsnufft_plan_last_error", "dfsnufft_es_kernel",
                            "dfsnufft_version"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _strerror(status):
    try:
        return lib().dfsnufft_strerror(int(status)).decode()
    except Exception:   # library not loadable: still describe the code
        return "status %d" % status


def _check(rc, plan_handle=None):
    if rc != OK:
        detail = ""
        if plan_handle is not None:
            detail = (lib().dfsnufft_plan_last_error(plan_handle) or b"").decode()
        raise DfsError(rc, detail)


def _dtype_code(dtype) -> int:
    if dtype in (F64, "f64", "float64", "double", np.float64):
        return F64
    if dtype in (F32, "f32", "float32", "float", np.float32):
        return F32
    raise ValueError("dtype must be 'f64' or 'f32'")


# ------------------------------------------------------------ host-only helpers

def dfsnufft_choose_params(n_lon, n_lat, tol, dtype="f64", options=None) -> dict:
    p = Params()
    if options is None:
        _check(lib().dfsnufft_choose_params(int(n_lon), int(n_lat), float(tol),
                                            _dtype_code(dtype), ctypes.byref(p)))
    else:
        _check(lib().dfsnufft_choose_params_opts(int(n_lon), int(n_lat), float(tol),
                                                 _dtype_code(dtype), ctypes.byref(options),
                                                 ctypes.byref(p)))
    return p.as_dict()


def dfsnufft_es_kernel(z, w, beta) -> float:
    return float(lib().dfsnufft_es_kernel(float(z), int(w), float(beta)))


def dfsnufft_kernel_ft(w, beta, n_fine, n_modes) -> np.ndarray:
    out = np.empty(int(n_modes), dtype=np.float64)
    _check(lib().dfsnufft_kernel_ft(int(w), float(beta), int(n_fine), int(n_modes),
                                    out.ctypes.data))
    return out


def dfsnufft_es_horner(w, beta) -> np.ndarray:
    """(w, w + 1) polynomial coefficients of the kernel taps in s = t - mid."""
    out = np.empty(int(w) * (int(w) + 1), dtype=np.float64)
    _check(lib().dfsnufft_es_horner(int(w), float(beta), out.ctypes.data))
    return out.reshape(int(w), int(w) + 1)


def dfsnufft_version() -> str:
    return lib().dfsnufft_version().decode()


# ------------------------------------------------------------ plan-level calls

def dfsnufft_plan_create(n_lon, n_lat, tol, dtype, n_fields, stream) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().dfsnufft_plan_create(int(n_lon), int(n_lat), float(tol), _dtype_code(dtype),
                                      int(n_fields), ctypes.c_void_p(int(stream or 0)),
                                      ctypes.byref(h)))
    return h


def dfsnufft_plan_create_batch(n_members, n_lon, n_lat, tol, dtype, n_fields, stream):
    h = ctypes.c_void_p()
    _check(lib().dfsnufft_plan_create_batch(int(n_members), int(n_lon), int(n_lat), float(tol),
                                            _dtype_code(dtype), int(n_fields),
                                            ctypes.c_void_p(int(stream or 0)), ctypes.byref(h)))
    return h


def dfsnufft_plan_create_opts(n_members, n_lon, n_lat, tol, dtype, n_fields, options, stream):
    h = ctypes.c_void_p()
    _check(lib().dfsnufft_plan_create_opts(int(n_members), int(n_lon), int(n_lat), float(tol),
                                           _dtype_code(dtype), int(n_fields),
                                           ctypes.byref(options) if options is not None else None,
                                           ctypes.c_void_p(int(stream or 0)), ctypes.byref(h)))
    return h


def dfsnufft_set_points_batch(h, counts, lon_ptr, colat_ptr):
    c = np.ascontiguousarray(counts, dtype=np.int64)
    _check(lib().dfsnufft_set_points_batch(h, c.ctypes.data, ctypes.c_void_p(lon_ptr),
                                           ctypes.c_void_p(colat_ptr)), h)


def dfsnufft_set_points(h, n_points, lon_ptr, colat_ptr):
    _check(lib().dfsnufft_set_points(h, int(n_points), ctypes.c_void_p(lon_ptr),
                                     ctypes.c_void_p(colat_ptr)), h)


def dfsnufft_execute(h, coeffs_ptr, values_ptr):
    _check(lib().dfsnufft_execute(h, ctypes.c_void_p(coeffs_ptr), ctypes.c_void_p(values_ptr)), h)


def dfsnufft_set_points_host(h, n_points, lon_ptr, colat_ptr):
    _check(lib().dfsnufft_set_points_host(h, int(n_points), ctypes.c_void_p(lon_ptr),
                                          ctypes.c_void_p(colat_ptr)), h)


def dfsnufft_execute_host(h, coeffs_ptr, values_ptr):
    _check(lib().dfsnufft_execute_host(h, ctypes.c_void_p(coeffs_ptr),
                                       ctypes.c_void_p(values_ptr)), h)


def dfsnufft_execute_points_host(h, n_points, lon_ptr, colat_ptr, coeffs_ptr, values_ptr):
    _check(lib().dfsnufft_execute_points_host(h, ctypes.c_int64(n_points), ctypes.c_void_p(lon_ptr),
                                              ctypes.c_void_p(colat_ptr),
                                              ctypes.c_void_p(coeffs_ptr),
                                              ctypes.c_void_p(values_ptr)), h)


def dfsnufft_destroy(h):
    _check(lib().dfsnufft_destroy(h))


def dfsnufft_plan_check(h):
    """Synchronise and raise DfsError if the plan (or a kernel of it) failed."""
    _check(lib().dfsnufft_plan_check(h), h)


def dfsnufft_plan_enable_timing(h, enable=True):
    _check(lib().dfsnufft_plan_enable_timing(h, 1 if enable else 0), h)


def dfsnufft_plan_read_timing(h) -> dict:
    """{stage: (total ms, calls)} for the stages of STAGES (synchronises)."""
    ms = np.zeros(N_STAGES, dtype=np.float64)
    calls = np.zeros(N_STAGES, dtype=np.int64)
    _check(lib().dfsnufft_plan_read_timing(h, ms.ctypes.data, calls.ctypes.data), h)
    return {STAGES[i]: (float(ms[i]), int(calls[i])) for i in range(N_STAGES)}


def dfsnufft_plan_point_stats(h) -> dict:
    rows = ctypes.c_int64()
    bins = ctypes.c_int64()
    _check(lib().dfsnufft_plan_point_stats(h, ctypes.byref(rows), ctypes.byref(bins)), h)
    return {"rows_needed": rows.value, "nonempty_bins": bins.value}


def dfsnufft_plan_host_copy_bytes(h) -> dict:
    pts, cf, vals = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().dfsnufft_plan_host_copy_bytes(h, ctypes.byref(pts), ctypes.byref(cf),
                                               ctypes.byref(vals)), h)
    return {"points_h2d": pts.value, "coeffs_h2d": cf.value, "values_d2h": vals.value}


def dfsnufft_probe_fma_rate(dtype, target_ms=20.0) -> float:
    out = ctypes.c_double()
    _check(lib().dfsnufft_probe_fma_rate(_dtype_code(dtype), float(target_ms), ctypes.byref(out)))
    return out.value


def dfsnufft_selftest_wait_timeout(cycles):
    """(device status word, kernel ms) of a bounded wait on a barrier nothing
    completes; status 1 means the wait gave up as designed."""
    st = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib().dfsnufft_selftest_wait_timeout(int(cycles), ctypes.byref(st), ctypes.byref(ms)))
    return st.value, ms.value


def dfsnufft_execute_noalloc(n_lon, n_lat, tol, dtype, n_fields, n_points, lon_ptr, colat_ptr,
                             coeffs_ptr, values_ptr, stream=0):
    """One-shot evaluation on the library's static device scratch: no device
    memory is allocated (for callers that cannot call cudaMalloc)."""
    _check(lib().dfsnufft_execute_noalloc(int(n_lon), int(n_lat), float(tol), _dtype_code(dtype),
                                          int(n_fields), int(n_points), ctypes.c_void_p(lon_ptr),
                                          ctypes.c_void_p(colat_ptr), ctypes.c_void_p(coeffs_ptr),
                                          ctypes.c_void_p(values_ptr),
                                          ctypes.c_void_p(int(stream or 0))))


def _stream_ptr(tensor, stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(tensor.device)
    return ctypes.c_void_p(int(stream.cuda_stream))


def _real_code(tensor) -> int:
    import torch
    if tensor.dtype == torch.float64:
        return F64
    if tensor.dtype == torch.float32:
        return F32
    raise TypeError("expected a float32 or float64 tensor, got %s" % tensor.dtype)


def departure_points(w, dt_over_a, iterations, w_arrival=None, stream=None, lon_out=None,
                     colat_out=None, pq_out=None):
    """Departure points (lon, colat) of Eq. 2.4 for every Grid [0] arrival point
    (dfsnufft_departure_points).  ``w``, ``w_arrival``: CUDA tensors of shape
    ([members,] 2, n_lat, n_lon), eastward then northward component; returns two
    float64 tensors of shape ([members,] n_lat * n_lon) (or fills the given ones).
    ``pq_out`` (optional, w's dtype, ([members,] 2, n_lat * n_lon) elements)
    receives p and q of the rotation to the arrival frame."""
    import torch
    if not w.is_cuda or not w.is_contiguous() or w.dim() not in (3, 4) or w.shape[-3] != 2:
        raise ValueError("w must be a contiguous CUDA tensor of shape ([members,] 2, n_lat, n_lon)")
    if w_arrival is not None and (w_arrival.shape != w.shape or w_arrival.dtype != w.dtype
                                  or not w_arrival.is_contiguous()):
        raise ValueError("w_arrival must match w in shape, dtype and layout")
    members = w.shape[0] if w.dim() == 4 else 1
    n_lat, n_lon = int(w.shape[-2]), int(w.shape[-1])
    shape = (members, n_lat * n_lon) if w.dim() == 4 else (n_lat * n_lon,)
    lon = torch.empty(shape, dtype=torch.float64, device=w.device) if lon_out is None else lon_out
    colat = (torch.empty(shape, dtype=torch.float64, device=w.device) if colat_out is None
             else colat_out)
    for t in (lon, colat):
        if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != members * n_lat * n_lon:
            raise ValueError("lon_out / colat_out: contiguous float64, one value per arrival point")
    if pq_out is not None and (pq_out.dtype != w.dtype or not pq_out.is_contiguous()
                               or pq_out.numel() != 2 * members * n_lat * n_lon):
        raise ValueError("pq_out: contiguous, w's dtype, two values per arrival point")
    _check(lib().dfsnufft_departure_points(
        n_lon, n_lat, members, _real_code(w), int(iterations), float(dt_over_a),
        ctypes.c_void_p(w.data_ptr()),
        ctypes.c_void_p(w_arrival.data_ptr() if w_arrival is not None else 0),
        ctypes.c_void_p(lon.data_ptr()), ctypes.c_void_p(colat.data_ptr()),
        ctypes.c_void_p(pq_out.data_ptr() if pq_out is not None else 0),
        _stream_ptr(w, stream)))
    return lon, colat


def rotate_to_arrival(n_lon, n_lat, lon_d, colat_d, u_d, v_d, stride=None, members=1,
                      u_a=None, v_a=None, stream=None, pq=None):
    """(u, v) at the departure points in the arrival points' frame
    (dfsnufft_rotate_to_arrival); u_d, v_d may be views into one values tensor,
    member m's point p at element m * stride + p.  With ``pq`` from
    :func:`departure_points` the rotation is read instead of computed from
    (lon_d, colat_d), which may then be None.  Returns (u_a, v_a); pass
    u_a = u_d, v_a = v_d to rotate in place."""
    import torch
    if stride is None:
        stride = n_lon * n_lat
    if u_a is None:
        u_a = torch.empty_like(u_d)
    if v_a is None:
        v_a = torch.empty_like(v_d)
    code = _real_code(u_d)
    for t in (v_d, u_a, v_a):
        if t.dtype != u_d.dtype or not t.is_cuda:
            raise ValueError("u_d, v_d, u_a, v_a must be CUDA tensors of one dtype")
    _check(lib().dfsnufft_rotate_to_arrival(
        int(n_lon), int(n_lat), int(members), code,
        ctypes.c_void_p(lon_d.data_ptr() if lon_d is not None else 0),
        ctypes.c_void_p(colat_d.data_ptr() if colat_d is not None else 0),
        ctypes.c_void_p(pq.data_ptr() if pq is not None else 0), ctypes.c_void_p(u_d.data_ptr()),
        ctypes.c_void_p(v_d.data_ptr()), int(stride), ctypes.c_void_p(u_a.data_ptr()),
        ctypes.c_void_p(v_a.data_ptr()), _stream_ptr(u_d, stream)))
    return u_a, v_a


def lagrange_interp(samples, parity, lon, colat, order, out=None, stream=None):
    """Cubic (order 3) or quintic (order 5) tensor Lagrange interpolation of
    Grid [0] samples, CUDA tensor (n_fields, n_lat, n_lon), at the points (lon,
    colat) (dfsnufft_lagrange_interp); returns (n_fields, n_points)."""
    import torch
    if not samples.is_cuda or not samples.is_contiguous() or samples.dim() != 3:
        raise ValueError("samples must be a contiguous CUDA tensor (n_fields, n_lat, n_lon)")
    F, n_lat, n_lon = (int(x) for x in samples.shape)
    par = np.ascontiguousarray(parity, dtype=np.int32)
    if par.size != F:
        raise ValueError("one parity per field")
    P = int(lon.numel())
    if out is None:
        out = torch.empty((F, P), dtype=samples.dtype, device=samples.device)
    _check(lib().dfsnufft_lagrange_interp(
        n_lon, n_lat, F, par.ctypes.data, int(order), _real_code(samples), P,
        ctypes.c_void_p(lon.data_ptr()), ctypes.c_void_p(colat.data_ptr()),
        ctypes.c_void_p(samples.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        _stream_ptr(samples, stream)))
    return out


def dfsnufft_plan_get_params(h) -> dict:
    p = Params()
    _check(lib().dfsnufft_plan_get_params(h, ctypes.byref(p)), h)
    return p.as_dict()


class Plan:
    """A type-2 NUFFT plan for an n_lat x n_lon grid (coefficients (F, 2 n_lat, n_lon)).

    ``set_points`` takes CUDA float64 tensors; ``execute`` takes a CUDA complex
    tensor (complex128 for 'f64', complex64 for 'f32') and returns or fills a
    (F, P) real tensor.  Work is enqueued on ``stream`` (default: torch's
    current stream at creation).  With ``n_members`` > 1 the plan is batched:
    coefficients (members, F, 2 n_lat, n_lon), points given per member
    (``set_points(lon, colat, counts)`` with concatenated arrays), values
    concatenated per member (each F x P_k).  ``options`` (an :class:`Options`)
    sets the real-field mode, oversampling, kernel width and bin size.
    """

    def __init__(self, n_lon, n_lat, tol=1e-12, dtype="f64", n_fields=1, stream=None,
                 n_members=1, options=None):
        import torch
        self.n_lon, self.n_lat = int(n_lon), int(n_lat)
        self.dtype = "f64" if _dtype_code(dtype) == F64 else "f32"
        self.n_fields = int(n_fields)
        self.n_members = int(n_members)
        self.tol = float(tol)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if options is not None:
            self._h = dfsnufft_plan_create_opts(self.n_members, n_lon, n_lat, tol, self.dtype,
                                                n_fields, options, handle)
        elif self.n_members == 1:
            self._h = dfsnufft_plan_create(n_lon, n_lat, tol, self.dtype, n_fields, handle)
        else:
            self._h = dfsnufft_plan_create_batch(self.n_members, n_lon, n_lat, tol, self.dtype,
                                                 n_fields, handle)
        self.params = dfsnufft_plan_get_params(self._h)
        self.n_points = 0
        self.counts = None
        self._keep = None

    @property
    def coeff_shape(self):
        if self.n_members == 1:
            return (self.n_fields, 2 * self.n_lat, self.n_lon)
        return (self.n_members, self.n_fields, 2 * self.n_lat, self.n_lon)

    def _real_dtype(self):
        import torch
        return torch.float64 if self.dtype == "f64" else torch.float32

    def _cplx_dtype(self):
        import torch
        return torch.complex128 if self.dtype == "f64" else torch.complex64

    def set_points(self, lon, colat, counts=None):
        import torch
        for t in (lon, colat):
            if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 1 and t.is_contiguous()):
                raise ValueError("points must be contiguous 1-D CUDA float64 tensors")
        if lon.numel() != colat.numel():
            raise ValueError("lon and colat differ in length")
        if counts is None:
            if self.n_members != 1:
                raise ValueError("a batched plan needs the per-member point counts")
            counts = [lon.numel()]
        counts = [int(c) for c in counts]
        if len(counts) != self.n_members or sum(counts) != lon.numel():
            raise ValueError("counts must give every member's points and sum to the total")
        dfsnufft_set_points_batch(self._h, counts, lon.data_ptr(), colat.data_ptr())
        self.n_points = lon.numel()
        self.counts = counts
        self._keep = (lon, colat)

    def execute(self, coeffs, out=None):
        import torch
        if tuple(coeffs.shape) != self.coeff_shape or coeffs.dtype != self._cplx_dtype() \
                or not coeffs.is_cuda or not coeffs.is_contiguous():
            raise ValueError("coeffs must be a contiguous CUDA %s tensor of shape %s"
                             % (self._cplx_dtype(), self.coeff_shape))
        shape = (self.n_fields, self.n_points) if self.n_members == 1 else \
            (self.n_fields * self.n_points,)
        if out is None:
            out = torch.empty(shape, dtype=self._real_dtype(), device=coeffs.device)
        elif out.numel() != self.n_fields * self.n_points or \
                out.dtype != self._real_dtype() or not out.is_contiguous():
            raise ValueError("out must be a contiguous %s tensor of %d values"
                             % (self._real_dtype(), self.n_fields * self.n_points))
        dfsnufft_execute(self._h, coeffs.data_ptr(), out.data_ptr())
        return out

    def execute_pr(self, pr, out=None):
        """Fields given by partial-regularity DFS coefficients (Sec. 4): ``pr`` a
        contiguous CUDA complex tensor of shape ([members,] F, M + 1, N + 1) with
        pr[..., m, n] = f^c_{n,m} + i f^s_{n,m}; the plan must be a real-field plan."""
        import torch
        lead = (self.n_fields,) if self.n_members == 1 else (self.n_members, self.n_fields)
        if tuple(pr.shape[:-2]) != lead or pr.dtype != self._cplx_dtype() or not pr.is_cuda \
                or not pr.is_contiguous() or pr.dim() != len(lead) + 2:
            raise ValueError("pr must be a contiguous CUDA %s tensor of shape %s + (M+1, N+1)"
                             % (self._cplx_dtype(), lead))
        M, N = pr.shape[-2] - 1, pr.shape[-1] - 1
        shape = (self.n_fields, self.n_points) if self.n_members == 1 else \
            (self.n_fields * self.n_points,)
        if out is None:
            out = torch.empty(shape, dtype=self._real_dtype(), device=pr.device)
        _check(lib().dfsnufft_execute_pr(self._h, int(M), int(N), ctypes.c_void_p(pr.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr())), self._h)
        return out

    def _grid_args(self, samples, parity):
        lead = (self.n_fields,) if self.n_members == 1 else (self.n_members, self.n_fields)
        if tuple(samples.shape) != lead + (self.n_lat, self.n_lon) or \
                samples.dtype != self._real_dtype() or not samples.is_cuda or \
                not samples.is_contiguous():
            raise ValueError("samples must be a contiguous CUDA %s tensor of shape %s"
                             % (self._real_dtype(), lead + (self.n_lat, self.n_lon)))
        par = np.ascontiguousarray(parity, dtype=np.int32)
        if par.shape != (self.n_fields,):
            raise ValueError("parity needs one entry (+1 or -1) per field")
        return par

    def latitudes(self):
        """Colatitudes of the arrival grid's rows (Gauss-Legendre nodes for a
        DFSNUFFT_GAUSS_GRID plan)."""
        out = np.empty(self.n_lat, dtype=np.float64)
        _check(lib().dfsnufft_plan_latitudes(self._h, out.ctypes.data), self._h)
        return out

    def grid_to_coeffs(self, samples, parity, out=None):
        """Coefficients (the execute layout) of fields sampled on the arrival grid
        (Grid [0]); parity +1 for scalars, -1 for wind components."""
        import torch
        par = self._grid_args(samples, parity)
        if out is None:
            out = torch.empty(self.coeff_shape, dtype=self._cplx_dtype(), device=samples.device)
        _check(lib().dfsnufft_grid_to_coeffs(self._h, ctypes.c_void_p(samples.data_ptr()),
                                             par.ctypes.data, ctypes.c_void_p(out.data_ptr())),
               self._h)
        return out

    def interpolate_grid(self, samples, parity, out=None):
        """Values at the plan's points of fields sampled on the arrival grid."""
        import torch
        par = self._grid_args(samples, parity)
        shape = (self.n_fields, self.n_points) if self.n_members == 1 else \
            (self.n_fields * self.n_points,)
        if out is None:
            out = torch.empty(shape, dtype=self._real_dtype(), device=samples.device)
        _check(lib().dfsnufft_interpolate_grid(self._h, ctypes.c_void_p(samples.data_ptr()),
                                               par.ctypes.data, ctypes.c_void_p(out.data_ptr())),
               self._h)
        return out

    def split_values(self, out):
        """Per-member (F, P_k) views of a batched plan's output."""
        views, o = [], 0
        for c in self.counts:
            views.append(out[o:o + self.n_fields * c].view(self.n_fields, c))
            o += self.n_fields * c
        return views

    def set_points_host(self, lon, colat):
        lon = np.ascontiguousarray(lon, dtype=np.float64)
        colat = np.ascontiguousarray(colat, dtype=np.float64)
        if lon.shape != colat.shape or lon.ndim != 1:
            raise ValueError("points must be 1-D float64 arrays of equal length")
        dfsnufft_set_points_host(self._h, lon.size, lon.ctypes.data, colat.ctypes.data)
        self.n_points = lon.size

    def execute_host(self, coeffs, out=None):
        cd = np.complex128 if self.dtype == "f64" else np.complex64
        rd = np.float64 if self.dtype == "f64" else np.float32
        c = np.ascontiguousarray(coeffs, dtype=cd)
        if c.shape != self.coeff_shape:
            raise ValueError("coeffs must have shape %s" % (self.coeff_shape,))
        if out is None:
            out = np.empty((self.n_fields, self.n_points), dtype=rd)
        dfsnufft_execute_host(self._h, c.ctypes.data, out.ctypes.data)
        return out

    def execute_points_host(self, lon, colat, coeffs, out=None):
        """set_points_host then execute_host as one call (host arrays in and out),
        the copies and passes scheduled together."""
        lon = np.ascontiguousarray(lon, dtype=np.float64)
        colat = np.ascontiguousarray(colat, dtype=np.float64)
        if lon.shape != colat.shape or lon.ndim != 1:
            raise ValueError("points must be 1-D float64 arrays of equal length")
        cd = np.complex128 if self.dtype == "f64" else np.complex64
        rd = np.float64 if self.dtype == "f64" else np.float32
        c = np.ascontiguousarray(coeffs, dtype=cd)
        if c.shape != self.coeff_shape:
            raise ValueError("coeffs must have shape %s" % (self.coeff_shape,))
        if out is None:
            out = np.empty((self.n_fields, lon.size), dtype=rd)
        dfsnufft_execute_points_host(self._h, lon.size, lon.ctypes.data, colat.ctypes.data,
                                     c.ctypes.data, out.ctypes.data)
        self.n_points = lon.size
        return out

    def check(self):
        """Synchronise the plan's stream; raise DfsError on a recorded failure."""
        dfsnufft_plan_check(self._h)

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            dfsnufft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Ensemble:
    """Members on uneven grids: ``groups`` is a list of (n_members, n_lon, n_lat).
    ``run(points, coeffs, out)`` takes, per group, (lon, colat, counts) CUDA
    float64 tensors/list, a (members, F, 2 n_lat, n_lon) complex tensor and an
    output tensor of F x sum(counts) reals; the whole step is one CUDA graph."""

    def __init__(self, groups, tol=1e-6, dtype="f32", n_fields=3, stream=None, options=None,
                 persistent=False):
        import torch
        self.groups = [tuple(int(x) for x in g) for g in groups]
        self.dtype = "f64" if _dtype_code(dtype) == F64 else "f32"
        self.n_fields = int(n_fields)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        G = len(self.groups)
        ai = lambda xs: (ctypes.c_int * G)(*xs)
        h = ctypes.c_void_p()
        opts = None
        if options is not None:       # one Options per group
            if len(options) != G:
                raise ValueError("options must give one entry per group")
            opts = (Options * G)(*options)
        _check(lib().dfsnufft_ensemble_create_opts(
            G, ai([g[0] for g in self.groups]), ai([g[1] for g in self.groups]),
            ai([g[2] for g in self.groups]), float(tol), _dtype_code(dtype), self.n_fields,
            opts, ctypes.c_void_p(int(handle)), ctypes.byref(h)))
        self._h = h
        self._keep = None
        if persistent:
            self.set_persistent(True)

    def set_persistent(self, on):
        """One persistent launch per step for the transform and interpolation
        of all groups (on), or the fork/join graph of per-group plans (off)."""
        _check(lib().dfsnufft_ensemble_set_persistent(self._h, 1 if on else 0))

    def selftest_queue_timeout(self, cycles):
        """Status of the last persistent step relaunched with a queue wait that
        cannot complete (ERR_TIMEOUT is the expected outcome)."""
        return lib().dfsnufft_ensemble_selftest_queue_timeout(self._h, int(cycles))

    def plan_handle(self, g):
        h = ctypes.c_void_p()
        _check(lib().dfsnufft_ensemble_plan(self._h, int(g), ctypes.byref(h)))
        return h

    def run(self, points, coeffs, outs):
        G = len(self.groups)
        counts = [np.ascontiguousarray(p[2], dtype=np.int64) for p in points]
        cptr = (ctypes.c_void_p * G)(*[c.ctypes.data for c in counts])
        vp = lambda xs: (ctypes.c_void_p * G)(*[x.data_ptr() for x in xs])
        rc = lib().dfsnufft_ensemble_run(self._h, cptr, vp([p[0] for p in points]),
                                         vp([p[1] for p in points]), vp(coeffs), vp(outs))
        self._keep = (counts, points, coeffs, outs)
        if rc != OK:
            raise DfsError(rc)

    def check(self):
        rc = lib().dfsnufft_ensemble_check(self._h)
        if rc != OK:
            raise DfsError(rc)

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dfsnufft_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
