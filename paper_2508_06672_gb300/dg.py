"""Python binding of libdg (``include/dg.h``): argument marshalling only.

Every step of the hot path runs in the CUDA library. torch provides device
memory and streams. If the library is missing this module raises on use; it
never falls back to another implementation.

Two layers:

* ``dg_*`` functions with the C names and arguments (ctypes), raising
  :class:`DGError` on a non-zero status;
* :class:`Geolocator`, a context object over torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "DGError", "dg_grid", "dg_ephem", "dg_options", "dg_fix", "dg_peak", "dg_tuning", "lib", "library_path",
    "Batch",
    "dg_options_default", "dg_create", "dg_load_capture", "dg_cost_surface", "dg_argmax_refine",
    "dg_sync", "dg_destroy", "dg_last_error", "dg_grid_ecef", "dg_step_geometry", "dg_kernel_time",
    "dg_reset_counters", "dg_launch_count", "dg_abi_version", "dg_fp32_peak", "dg_debug_tc_wait_limit", "Geolocator",
    "dg_cost_surface_noalloc", "dg_noalloc_last_error", "DG_NOALLOC_SCRATCH_BYTES", "dg_cdft_work",
    "DG_OK", "DG_EINVAL", "DG_ENOMEM", "DG_ECUDA", "DG_ESTATE", "DG_ETIMEOUT", "DG_EUNSUPPORTED",
    "DG_IQ_C64", "DG_IQ_CI16", "DG_IQ_CI8", "DG_DELAY_INTEGER", "DG_DELAY_LAGRANGE4",
    "DG_ACC_POWER", "DG_ACC_MAG", "DG_PREC_FP32", "DG_PREC_FP64", "DG_ALGO_DIRECT", "DG_ALGO_CDFT",
    "DG_CONTRACT_FP32", "DG_CONTRACT_BF16", "DG_CONTRACT_FP16", "DG_CONTRACT_BF16X3", "DG_CONTRACT_FP16X3",
    "DG_K_CORR", "DG_K_ACCUM", "DG_K_ARGMAX", "DG_K_GRID", "DG_K_REFINE", "EXPORTED_SYMBOLS",
    "DG_K_CDFT_PLAN", "DG_K_CDFT_CONTRACT", "DG_K_CDFT_COMBINE",
    "dg_nn_conv3x3_forward", "dg_nn_conv3x3_backward", "dg_nn_relu_forward", "dg_nn_relu_backward",
    "dg_nn_bce_logits", "dg_nn_adam", "dg_nn_last_error", "dg_coarse_step", "DG_K_COARSE",
    "dg_nn_conv3x3_forward_tc", "dg_nn_conv3x3_backward_tc", "dg_nn_tc_check",
]

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ESTATE, DG_ETIMEOUT, DG_EUNSUPPORTED = range(7)
DG_IQ_C64, DG_IQ_CI16, DG_IQ_CI8 = 0, 1, 2
DG_DELAY_INTEGER, DG_DELAY_LAGRANGE4 = 0, 1
DG_ACC_POWER, DG_ACC_MAG = 0, 1
DG_PREC_FP32, DG_PREC_FP64 = 0, 1
DG_ALGO_DIRECT, DG_ALGO_CDFT = 0, 1
DG_CONTRACT_FP32, DG_CONTRACT_BF16, DG_CONTRACT_FP16, DG_CONTRACT_BF16X3, DG_CONTRACT_FP16X3 = 0, 1, 2, 3, 4
DG_TILES_AUTO, DG_TILES_ROWS, DG_TILES_LAGS, DG_TILES_HANKEL = 0, 1, 2, 3
DG_K_CORR, DG_K_ACCUM, DG_K_ARGMAX, DG_K_GRID, DG_K_REFINE = 0, 1, 2, 3, 4
DG_K_CDFT_PLAN, DG_K_CDFT_CONTRACT, DG_K_CDFT_COMBINE, DG_K_COARSE = 5, 6, 7, 8

_FMT = {"c64": DG_IQ_C64, "ci16": DG_IQ_CI16, "ci8": DG_IQ_CI8}
_FMT_DTYPE = {DG_IQ_C64: np.float32, DG_IQ_CI16: np.int16, DG_IQ_CI8: np.int8}
_DELAY = {"integer": DG_DELAY_INTEGER, "lagrange4": DG_DELAY_LAGRANGE4}
_ACC = {"power": DG_ACC_POWER, "mag": DG_ACC_MAG}
_PREC = {"fp32": DG_PREC_FP32, "fp64": DG_PREC_FP64}
_ALGO = {"direct": DG_ALGO_DIRECT, "cdft": DG_ALGO_CDFT}
_TILES = {"auto": DG_TILES_AUTO, "rows": DG_TILES_ROWS, "lags": DG_TILES_LAGS, "hankel": DG_TILES_HANKEL}
_CONTRACT = {"fp32": DG_CONTRACT_FP32, "bf16": DG_CONTRACT_BF16, "fp16": DG_CONTRACT_FP16,
             "bf16x3": DG_CONTRACT_BF16X3, "fp16x3": DG_CONTRACT_FP16X3}

EXPORTED_SYMBOLS = [
    "dg_options_default", "dg_create", "dg_load_capture", "dg_cost_surface", "dg_argmax_refine",
    "dg_sync", "dg_destroy", "dg_last_error", "dg_grid_ecef", "dg_step_geometry", "dg_kernel_time",
    "dg_reset_counters", "dg_launch_count", "dg_abi_version", "dg_cost_surface_noalloc",
    "dg_noalloc_last_error", "dg_cdft_work", "dg_detect", "dg_cdft_chunks",
    "dg_graph_capture", "dg_graph_launch", "dg_graph_fix", "dg_batch_capture", "dg_batch_launch",
    "dg_batch_fixes", "dg_batch_launch_count", "dg_batch_destroy", "dg_autotune",
    "dg_nn_conv3x3_forward", "dg_nn_conv3x3_backward", "dg_nn_conv3x3_scratch", "dg_nn_relu_forward",
    "dg_nn_relu_backward", "dg_nn_bce_scratch", "dg_nn_bce_logits", "dg_nn_adam", "dg_nn_last_error",
    "dg_coarse_maps", "dg_coarse_inspect", "dg_set_grid", "dg_search_regions", "dg_fp32_peak",
    "dg_debug_tc_wait_limit", "dg_batch_rounds", "dg_nn_conv3x3_forward_tc", "dg_nn_conv3x3_backward_tc",
    "dg_nn_conv3x3_tc_scratch", "dg_nn_tc_check",
]
DG_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


class DGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"dg status {status}: {message}")
        self.status = status


class dg_grid(C.Structure):
    _fields_ = [("lat0_deg", C.c_double), ("lon0_deg", C.c_double), ("dlat_m", C.c_double),
                ("dlon_m", C.c_double), ("nlat", C.c_int32), ("nlon", C.c_int32)]

    @classmethod
    def from_dict(cls, d):
        return cls(float(d["lat0_deg"]), float(d["lon0_deg"]), float(d["dlat_m"]),
                   float(d["dlon_m"]), int(d["nlat"]), int(d["nlon"]))


class dg_ephem(C.Structure):
    _fields_ = [("p1", C.c_double * 3), ("v1", C.c_double * 3), ("p2", C.c_double * 3),
                ("v2", C.c_double * 3)]


class dg_options(C.Structure):
    _fields_ = [("delay", C.c_int32), ("acc", C.c_int32), ("prec", C.c_int32), ("algo", C.c_int32),
                ("row0", C.c_int32), ("nrows", C.c_int32), ("timing", C.c_int32),
                ("chunk", C.c_int32), ("bins", C.c_int32), ("contract", C.c_int32),
                ("tiles", C.c_int32), ("scratch_mib", C.c_int32), ("rows", C.c_int32)]


class dg_tuning(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("tiles", C.c_int32), ("ms", C.c_double), ("tried", C.c_int32),
                ("cached", C.c_int32), ("rows", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dg_peak(C.Structure):
    _fields_ = [("index", C.c_int64), ("i", C.c_int32), ("j", C.c_int32), ("lat_deg", C.c_double),
                ("lon_deg", C.c_double), ("value", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dg_coarse_step(C.Structure):
    _fields_ = [("l0", C.c_int32), ("nlag", C.c_int32), ("nu_lo", C.c_double), ("delta", C.c_double),
                ("nu_c", C.c_double), ("mu", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dg_fix(C.Structure):
    _fields_ = [("index", C.c_int64), ("i", C.c_int32), ("j", C.c_int32), ("lat_deg", C.c_double),
                ("lon_deg", C.c_double), ("cost", C.c_double), ("refine_n", C.c_int32),
                ("ri", C.c_int32), ("rj", C.c_int32), ("pad", C.c_int32),
                ("refined_lat_deg", C.c_double), ("refined_lon_deg", C.c_double),
                ("refined_cost", C.c_double), ("sub_lat_deg", C.c_double), ("sub_lon_deg", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_LOCK = threading.Lock()
_LIB = None


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libdg.so")


def lib():
    """The loaded libdg.so; raises if it has not been built."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                                   "(needs nvcc); there is no fallback implementation")
            L = C.CDLL(path)
            vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            L.dg_options_default.argtypes = [C.POINTER(dg_options)]
            L.dg_options_default.restype = None
            L.dg_create.argtypes = [C.POINTER(dg_grid), C.POINTER(dg_ephem), i32, dbl, dbl,
                                    C.POINTER(dg_options), vp, C.POINTER(vp)]
            L.dg_load_capture.argtypes = [vp, i32, i32, vp, vp, i64, i32]
            L.dg_cost_surface.argtypes = [vp, vp]
            L.dg_argmax_refine.argtypes = [vp, vp, dbl, dbl, C.POINTER(dg_fix)]
            L.dg_sync.argtypes = [vp]
            L.dg_destroy.argtypes = [vp]
            L.dg_last_error.argtypes = [vp]
            L.dg_last_error.restype = C.c_char_p
            L.dg_grid_ecef.argtypes = [vp, vp]
            L.dg_step_geometry.argtypes = [vp, i32, vp, vp, vp]
            L.dg_kernel_time.argtypes = [vp, i32, C.POINTER(dbl), C.POINTER(i64)]
            L.dg_reset_counters.argtypes = [vp]
            L.dg_launch_count.argtypes = [vp]
            L.dg_launch_count.restype = i64
            L.dg_abi_version.argtypes = []
            L.dg_abi_version.restype = i32
            L.dg_fp32_peak.argtypes = [vp, i32, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(i32)]
            L.dg_debug_tc_wait_limit.argtypes = [C.c_uint32]
            L.dg_cost_surface_noalloc.argtypes = [C.POINTER(dg_grid), C.POINTER(dg_ephem), i32, dbl, dbl,
                                                  i32, vp, vp, i64, C.POINTER(dg_options), vp, vp]
            L.dg_cost_surface_noalloc.restype = C.c_int
            L.dg_detect.argtypes = [vp, vp, dbl, i32, i32, i32, C.POINTER(dg_peak), C.POINTER(i32)]
            L.dg_detect.restype = C.c_int
            L.dg_graph_capture.argtypes = [vp, vp, dbl, dbl]
            L.dg_graph_launch.argtypes = [vp]
            L.dg_graph_fix.argtypes = [vp, C.POINTER(dg_fix)]
            L.dg_batch_capture.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), dbl, dbl, vp, C.POINTER(vp)]
            L.dg_batch_launch.argtypes = [vp]
            L.dg_batch_fixes.argtypes = [vp, C.POINTER(dg_fix)]
            L.dg_batch_launch_count.argtypes = [vp]
            L.dg_batch_launch_count.restype = C.c_int64
            L.dg_batch_destroy.argtypes = [vp]
            L.dg_batch_rounds.argtypes = [vp]
            L.dg_batch_rounds.restype = i32
            for f in ("dg_graph_capture", "dg_graph_launch", "dg_graph_fix", "dg_batch_capture", "dg_batch_launch",
                      "dg_batch_fixes", "dg_batch_destroy"):
                getattr(L, f).restype = C.c_int
            L.dg_autotune.argtypes = [vp, vp, i32, C.POINTER(dg_tuning)]
            L.dg_autotune.restype = C.c_int
            L.dg_cdft_chunks.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
            L.dg_cdft_chunks.restype = C.c_int
            L.dg_cdft_work.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
            L.dg_cdft_work.restype = C.c_int
            L.dg_noalloc_last_error.argtypes = []
            L.dg_noalloc_last_error.restype = C.c_char_p
            flt = C.c_float
            L.dg_search_regions.argtypes = [vp, C.POINTER(dg_grid), i32, vp, dbl, dbl, C.POINTER(dg_fix),
                                            C.POINTER(i32)]
            L.dg_search_regions.restype = C.c_int
            L.dg_set_grid.argtypes = [vp, C.POINTER(dg_grid)]
            L.dg_set_grid.restype = C.c_int
            L.dg_coarse_maps.argtypes = [vp, i32, i32, vp]
            L.dg_coarse_maps.restype = C.c_int
            L.dg_coarse_inspect.argtypes = [vp, vp, C.POINTER(dg_coarse_step), C.POINTER(i32)]
            L.dg_coarse_inspect.restype = C.c_int
            L.dg_nn_conv3x3_forward.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp]
            L.dg_nn_conv3x3_backward.argtypes = [vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
            L.dg_nn_conv3x3_scratch.argtypes = [i32, i32, i32, i32, i32]
            L.dg_nn_conv3x3_scratch.restype = i64
            L.dg_nn_conv3x3_forward_tc.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
            L.dg_nn_conv3x3_backward_tc.argtypes = [vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
            L.dg_nn_conv3x3_tc_scratch.argtypes = [i32, i32, i32, i32, i32]
            L.dg_nn_conv3x3_tc_scratch.restype = i64
            L.dg_nn_tc_check.argtypes = [vp]
            L.dg_nn_relu_forward.argtypes = [vp, vp, i64, vp]
            L.dg_nn_relu_backward.argtypes = [vp, vp, vp, i64, vp]
            L.dg_nn_bce_scratch.argtypes = [i64]
            L.dg_nn_bce_scratch.restype = i64
            L.dg_nn_bce_logits.argtypes = [vp, vp, flt, i64, vp, vp, vp, vp]
            L.dg_nn_adam.argtypes = [vp, vp, vp, vp, i64, flt, flt, flt, flt, i32, vp]
            for f in ("dg_nn_conv3x3_forward", "dg_nn_conv3x3_backward", "dg_nn_relu_forward",
                      "dg_nn_relu_backward", "dg_nn_bce_logits", "dg_nn_adam", "dg_nn_conv3x3_forward_tc",
                      "dg_nn_conv3x3_backward_tc", "dg_nn_tc_check"):
                getattr(L, f).restype = C.c_int
            L.dg_nn_last_error.argtypes = []
            L.dg_nn_last_error.restype = C.c_char_p
            for name in ("dg_create", "dg_load_capture", "dg_cost_surface", "dg_argmax_refine",
                         "dg_sync", "dg_destroy", "dg_grid_ecef", "dg_step_geometry",
                         "dg_kernel_time", "dg_reset_counters"):
                getattr(L, name).restype = C.c_int
            _LIB = L
    return _LIB


def _check(status, ctx=None):
    if status != DG_OK:
        msg = lib().dg_last_error(ctx)
        raise DGError(status, msg.decode() if msg else "")


# ----------------------------------------------------------------- C names
def dg_options_default():
    o = dg_options()
    lib().dg_options_default(C.byref(o))
    return o


def dg_create(grid, ephem, K, fs_hz, fc_hz, opt=None, stream=0):
    """grid: dg_grid or dict; ephem: (K, 12) float64 array [p1 v1 p2 v2]."""
    g = grid if isinstance(grid, dg_grid) else dg_grid.from_dict(grid)
    eph = np.ascontiguousarray(ephem, dtype=np.float64).reshape(-1, 12)
    arr = (dg_ephem * max(1, eph.shape[0]))()
    C.memmove(arr, eph.ctypes.data, eph.nbytes)
    out = C.c_void_p()
    st = lib().dg_create(C.byref(g), arr, int(K), float(fs_hz), float(fc_hz),
                         C.byref(opt) if opt is not None else None, C.c_void_p(int(stream)),
                         C.byref(out))
    _check(st, None)
    return out.value


def dg_load_capture(ctx, step, fmt, y1_ptr, y2_ptr, n_samples, is_device_ptr):
    _check(lib().dg_load_capture(ctx, int(step), int(fmt), C.c_void_p(y1_ptr), C.c_void_p(y2_ptr),
                                 int(n_samples), int(is_device_ptr)), ctx)


def dg_cost_surface(ctx, out_ptr):
    _check(lib().dg_cost_surface(ctx, C.c_void_p(out_ptr)), ctx)


def dg_argmax_refine(ctx, cost_ptr, refine_spacing_m=0.0, window_m=0.0):
    f = dg_fix()
    _check(lib().dg_argmax_refine(ctx, C.c_void_p(cost_ptr), float(refine_spacing_m),
                                  float(window_m), C.byref(f)), ctx)
    return f


def dg_sync(ctx):
    _check(lib().dg_sync(ctx), ctx)


def dg_destroy(ctx):
    _check(lib().dg_destroy(ctx), None)


def dg_last_error(ctx=None):
    m = lib().dg_last_error(ctx)
    return m.decode() if m else ""


def dg_grid_ecef(ctx, xyz_ptr):
    _check(lib().dg_grid_ecef(ctx, C.c_void_p(xyz_ptr)), ctx)


def dg_step_geometry(ctx, step, lag_ptr=0, D_ptr=0, nu_ptr=0):
    _check(lib().dg_step_geometry(ctx, int(step), C.c_void_p(lag_ptr or None),
                                  C.c_void_p(D_ptr or None), C.c_void_p(nu_ptr or None)), ctx)


def dg_kernel_time(ctx, kernel_class):
    ms, n = C.c_double(), C.c_int64()
    _check(lib().dg_kernel_time(ctx, int(kernel_class), C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


class Batch:
    """Many Geolocator steps as one CUDA graph (dg_batch_*): each context's
    step -- surface into costs[i], argmax, refinement -- is a branch forked
    from and joined to `stream`; launch() enqueues all of them, fixes()
    waits and returns one fix per context."""

    def __init__(self, geolocators, costs, refine_spacing_m=0.0, refine_window_m=0.0, stream=None):
        import torch
        self.gs = list(geolocators)
        self.costs = list(costs)
        if len(self.gs) != len(self.costs) or not self.gs:
            raise ValueError("one cost tensor per geolocator")
        self.stream = stream if stream is not None else torch.cuda.Stream(self.gs[0].device)
        n = len(self.gs)
        ctxs = (C.c_void_p * n)(*[g.ctx for g in self.gs])
        ptrs = (C.c_void_p * n)(*[c.data_ptr() for c in self.costs])
        out = C.c_void_p()
        with torch.cuda.device(self.gs[0].device):
            st = lib().dg_batch_capture(ctxs, n, ptrs, float(refine_spacing_m), float(refine_window_m),
                                        C.c_void_p(self.stream.cuda_stream), C.byref(out))
        _check(st, None)
        self.handle = out

    def launch(self):
        _check(lib().dg_batch_launch(self.handle), None)

    def fixes(self):
        n = len(self.gs)
        arr = (dg_fix * n)()
        _check(lib().dg_batch_fixes(self.handle, arr), None)
        return [arr[i].as_dict() for i in range(n)]

    def launch_count(self):
        return int(lib().dg_batch_launch_count(self.handle))

    def rounds(self):
        """Shared contraction rounds of the batch (0: per-context launches)."""
        return int(lib().dg_batch_rounds(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().dg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_detect(ctx, cost_ptr, threshold, relative=False, radius=3, max_peaks=16):
    arr = (dg_peak * int(max_peaks))()
    n = C.c_int32()
    _check(lib().dg_detect(ctx, C.c_void_p(cost_ptr), float(threshold), int(bool(relative)), int(radius),
                           int(max_peaks), arr, C.byref(n)), ctx)
    return [arr[k].as_dict() for k in range(n.value)]


def dg_cdft_work(ctx):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().dg_cdft_work(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def dg_reset_counters(ctx):
    _check(lib().dg_reset_counters(ctx), ctx)


def dg_launch_count(ctx):
    return int(lib().dg_launch_count(ctx))


def dg_abi_version():
    return int(lib().dg_abi_version())


def dg_fp32_peak(iters=50000, stream=0):
    """Measured FP32 FMA throughput of the current device (see include/dg.h):
    returns (TFLOP/s, launch ms, SM count)."""
    tf, ms, sms = C.c_double(), C.c_double(), C.c_int32()
    st = lib().dg_fp32_peak(C.c_void_p(int(stream)), int(iters), C.byref(tf), C.byref(ms), C.byref(sms))
    if st != DG_OK:
        raise DGError(st, "dg_fp32_peak failed")
    return tf.value, ms.value, sms.value


def dg_debug_tc_wait_limit(polls):
    """Test hook (see include/dg.h): poll limit of the tensor-core pipeline's
    waits in CDFT surfaces launched afterwards; 0 restores the default."""
    lib().dg_debug_tc_wait_limit(int(polls))


def dg_noalloc_last_error():
    m = lib().dg_noalloc_last_error()
    return m.decode() if m else ""


def dg_cost_surface_noalloc(grid, ephem, fs_hz, fc_hz, fmt, y1_ptr, y2_ptr, n_samples, out_ptr,
                            opt=None, stream=0):
    """The allocation-free surface (see include/dg.h): captures y1/y2 and out
    are device pointers the caller owns; nothing is allocated on the device."""
    g = grid if isinstance(grid, dg_grid) else dg_grid.from_dict(grid)
    eph = np.ascontiguousarray(ephem, dtype=np.float64).reshape(-1, 12)
    arr = (dg_ephem * max(1, eph.shape[0]))()
    C.memmove(arr, eph.ctypes.data, eph.nbytes)
    st = lib().dg_cost_surface_noalloc(C.byref(g), arr, eph.shape[0], float(fs_hz), float(fc_hz),
                                       int(fmt), C.c_void_p(y1_ptr), C.c_void_p(y2_ptr), int(n_samples),
                                       C.byref(opt) if opt is not None else None, C.c_void_p(out_ptr),
                                       C.c_void_p(int(stream)))
    if st != DG_OK:
        raise DGError(st, dg_noalloc_last_error())


# ------------------------------------------------- proposal-network layers
# Thin marshalling over the dg_nn_* calls: torch CUDA tensors in (FP32,
# contiguous, NCHW), pointers and sizes out; the kernels do all the work.
def dg_nn_last_error():
    m = lib().dg_nn_last_error()
    return m.decode() if m else ""


def _nn_check(st):
    if st != DG_OK:
        raise DGError(st, dg_nn_last_error())


def _f32(*ts):
    for t in ts:
        if t is None:
            continue
        if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4 and t.is_contiguous()):
            raise ValueError("dg_nn_*: tensors must be contiguous float32 CUDA tensors")


def _ptr(t):
    return C.c_void_p(t.data_ptr() if t is not None else 0)


def _stream(stream, t):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return C.c_void_p(s.cuda_stream)


def dg_nn_conv3x3_forward(x, w, b, y, stream=None):
    """y = conv3x3(x, w) + b (NCHW; w: Co x Ci x 3 x 3)."""
    _f32(x, w, b, y)
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    if tuple(w.shape) != (Co, Ci, 3, 3) or tuple(b.shape) != (Co,) or tuple(y.shape) != (B, Co, H, W):
        raise ValueError("dg_nn_conv3x3_forward: shape mismatch")
    _nn_check(lib().dg_nn_conv3x3_forward(_ptr(x), _ptr(w), _ptr(b), _ptr(y), B, Ci, Co, H, W,
                                          _stream(stream, x)))


def dg_nn_conv3x3_backward(x, w, dy, dx, dw, db, scratch=None, stream=None):
    """Gradients of sum(dy * conv3x3(x, w, b)): dx (None: skipped), dw, db.
    scratch: dg_nn_conv3x3_scratch floats (allocated here when None)."""
    import torch
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    need = int(lib().dg_nn_conv3x3_scratch(B, Ci, Co, H, W))
    if need < 0:
        raise ValueError("dg_nn_conv3x3_backward: shape out of range")
    if scratch is None:
        scratch = torch.empty(max(1, need), dtype=torch.float32, device=x.device)
    _f32(x, w, dy, dx, dw, db, scratch)
    if (tuple(dy.shape) != (B, Co, H, W) or tuple(dw.shape) != (Co, Ci, 3, 3) or tuple(db.shape) != (Co,)
            or (dx is not None and tuple(dx.shape) != tuple(x.shape)) or scratch.numel() < need):
        raise ValueError("dg_nn_conv3x3_backward: shape mismatch")
    _nn_check(lib().dg_nn_conv3x3_backward(_ptr(x), _ptr(w), _ptr(dy), _ptr(dx), _ptr(dw), _ptr(db),
                                           B, Ci, Co, H, W, _ptr(scratch), _stream(stream, x)))


def dg_nn_conv3x3_forward_tc(x, w, b, y, scratch=None, stream=None):
    """dg_nn_conv3x3_forward on the tensor cores: BF16 operands, FP32 sums;
    scratch: dg_nn_conv3x3_tc_scratch floats (allocated here when None)."""
    import torch
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    need = int(lib().dg_nn_conv3x3_tc_scratch(B, Ci, Co, H, W))
    if need < 0:
        raise ValueError("dg_nn_conv3x3_forward_tc: shape out of range")
    if scratch is None:
        scratch = torch.empty(max(1, need), dtype=torch.float32, device=x.device)
    _f32(x, w, b, y, scratch)
    if (tuple(w.shape) != (Co, Ci, 3, 3) or tuple(b.shape) != (Co,) or tuple(y.shape) != (B, Co, H, W)
            or scratch.numel() < need):
        raise ValueError("dg_nn_conv3x3_forward_tc: shape mismatch")
    _nn_check(lib().dg_nn_conv3x3_forward_tc(_ptr(x), _ptr(w), _ptr(b), _ptr(y), B, Ci, Co, H, W,
                                             _ptr(scratch), _stream(stream, x)))


def dg_nn_conv3x3_backward_tc(x, w, dy, dx, dw, db, scratch=None, stream=None):
    """dg_nn_conv3x3_backward on the tensor cores: BF16 operands, FP32 sums;
    scratch: dg_nn_conv3x3_tc_scratch floats (allocated here when None)."""
    import torch
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    need = int(lib().dg_nn_conv3x3_tc_scratch(B, Ci, Co, H, W))
    if need < 0:
        raise ValueError("dg_nn_conv3x3_backward_tc: shape out of range")
    if scratch is None:
        scratch = torch.empty(max(1, need), dtype=torch.float32, device=x.device)
    _f32(x, w, dy, dx, dw, db, scratch)
    if (tuple(dy.shape) != (B, Co, H, W) or tuple(dw.shape) != (Co, Ci, 3, 3) or tuple(db.shape) != (Co,)
            or (dx is not None and tuple(dx.shape) != tuple(x.shape)) or scratch.numel() < need):
        raise ValueError("dg_nn_conv3x3_backward_tc: shape mismatch")
    _nn_check(lib().dg_nn_conv3x3_backward_tc(_ptr(x), _ptr(w), _ptr(dy), _ptr(dx), _ptr(dw), _ptr(db),
                                              B, Ci, Co, H, W, _ptr(scratch), _stream(stream, x)))


def dg_nn_tc_check(stream=None):
    """Raises DGError(DG_ETIMEOUT) if a tensor-core layer's wait ran out."""
    _nn_check(lib().dg_nn_tc_check(C.c_void_p(stream.cuda_stream if stream is not None else 0)))


def dg_nn_relu_forward(z, h, stream=None):
    _f32(z, h)
    if z.numel() != h.numel():
        raise ValueError("dg_nn_relu_forward: size mismatch")
    _nn_check(lib().dg_nn_relu_forward(_ptr(z), _ptr(h), z.numel(), _stream(stream, z)))


def dg_nn_relu_backward(z, dh, dz, stream=None):
    _f32(z, dh, dz)
    if not (z.numel() == dh.numel() == dz.numel()):
        raise ValueError("dg_nn_relu_backward: size mismatch")
    _nn_check(lib().dg_nn_relu_backward(_ptr(z), _ptr(dh), _ptr(dz), z.numel(), _stream(stream, z)))


def dg_nn_bce_logits(z, t, pos_weight, grad, loss, scratch=None, stream=None):
    """Mean weighted BCE on logits into loss (1 float) and its gradient into
    grad; scratch: dg_nn_bce_scratch(n) floats (allocated here when None)."""
    import torch
    n = z.numel()
    if scratch is None:
        scratch = torch.empty(max(1, int(lib().dg_nn_bce_scratch(n))), dtype=torch.float32, device=z.device)
    _f32(z, t, grad, loss, scratch)
    if not (t.numel() == n == grad.numel()) or loss.numel() < 1 or scratch.numel() < lib().dg_nn_bce_scratch(n):
        raise ValueError("dg_nn_bce_logits: size mismatch")
    _nn_check(lib().dg_nn_bce_logits(_ptr(z), _ptr(t), float(pos_weight), n, _ptr(grad), _ptr(loss),
                                     _ptr(scratch), _stream(stream, z)))


def dg_nn_adam(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step in place on p, m, v."""
    _f32(p, g, m, v)
    if not (p.numel() == g.numel() == m.numel() == v.numel()):
        raise ValueError("dg_nn_adam: size mismatch")
    _nn_check(lib().dg_nn_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), _stream(stream, p)))


# ------------------------------------------------------- torch-level object
class Geolocator:
    """One dg context: a grid (or a row shard of it), K snapshots, options.

    Device memory comes from torch; work runs on ``stream`` (a
    torch.cuda.Stream, default: the current stream of the device)."""

    def __init__(self, grid, ephem, fs_hz, fc_hz, *, delay="integer", acc="power", prec="fp32",
                 algo="direct", row0=0, nrows=0, timing=False, stream=None, device=None,
                 chunk=0, bins=0, contract="fp32", tiles="auto", scratch_mib=0, rows=0):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.grid = dict(grid)
        eph = np.ascontiguousarray(ephem, dtype=np.float64).reshape(-1, 12)
        self.K = eph.shape[0]
        self.opt = dg_options_default()
        self.opt.delay, self.opt.acc = _DELAY[delay], _ACC[acc]
        self.opt.prec, self.opt.algo = _PREC[prec], _ALGO[algo]
        self.opt.row0, self.opt.nrows, self.opt.timing = int(row0), int(nrows), int(bool(timing))
        self.opt.chunk, self.opt.bins, self.opt.contract = int(chunk), int(bins), _CONTRACT[contract]
        self.opt.tiles = _TILES[tiles]
        self.opt.scratch_mib = int(scratch_mib)
        self.opt.rows = int(rows)
        self.nrows = int(nrows) if nrows else int(grid["nlat"]) - int(row0)
        self.nlon = int(grid["nlon"])
        self.dtype = torch.float64 if prec == "fp64" else torch.float32
        self._keep = {}
        with torch.cuda.device(self.device):
            self.ctx = dg_create(self.grid, eph, self.K, fs_hz, fc_hz, self.opt, self.stream.cuda_stream)

    # -- captures
    def load_capture(self, step, fmt, y1, y2):
        """y1, y2: (N, 2) interleaved I/Q, as torch tensors (CUDA or host) or
        numpy arrays (host), of the storage type of fmt."""
        torch = self.torch
        code = _FMT[fmt] if isinstance(fmt, str) else int(fmt)
        ptrs, dev = [], None
        for y in (y1, y2):
            if isinstance(y, np.ndarray):
                y = torch.from_numpy(np.ascontiguousarray(y))
            if not y.is_contiguous():
                y = y.contiguous()
            if y.dtype != torch.from_numpy(np.zeros(1, _FMT_DTYPE[code])).dtype:
                raise TypeError(f"format {fmt} needs {_FMT_DTYPE[code].__name__} samples, got {y.dtype}")
            if y.dim() != 2 or y.shape[1] != 2:
                raise ValueError("captures must be (N, 2) interleaved I/Q")
            d = bool(y.is_cuda)
            if dev is not None and d != dev:
                raise ValueError("y1 and y2 must both be on the device or both on the host")
            dev = d
            ptrs.append(y)
        if ptrs[0].shape != ptrs[1].shape:
            raise ValueError("y1 and y2 must have the same number of samples")
        self._keep[step] = ptrs  # keep host buffers alive until the copy is ordered
        dg_load_capture(self.ctx, step, code, ptrs[0].data_ptr(), ptrs[1].data_ptr(), ptrs[0].shape[0],
                        1 if dev else 0)

    def load_captures(self, fmt, y1, y2):
        """All K snapshots: y1, y2 of shape (K, N, 2)."""
        for k in range(self.K):
            self.load_capture(k, fmt, y1[k], y2[k])

    # -- the hot path
    def cost_surface(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((self.nrows, self.nlon), dtype=self.dtype, device=self.device)
        if out.dtype != self.dtype or not out.is_cuda or not out.is_contiguous() or out.numel() < self.nrows * self.nlon:
            raise ValueError("out must be a contiguous CUDA tensor of the context's precision")
        dg_cost_surface(self.ctx, out.data_ptr())
        return out

    def argmax_refine(self, cost, refine_spacing_m=0.0, window_m=0.0):
        if cost.dtype != self.dtype or not cost.is_cuda:
            raise ValueError("cost must be a CUDA tensor of the context's precision")
        return dg_argmax_refine(self.ctx, cost.data_ptr(), refine_spacing_m, window_m).as_dict()

    def autotune(self, cost=None, reps=3):
        """Time the admissible launch shapes (CDFT: chunk and tiles; DIRECT:
        grid rows per thread) and keep the fastest."""
        if cost is None:
            cost = self.torch.empty((self.nrows, self.nlon), dtype=self.dtype, device=self.device)
        t = dg_tuning()
        _check(lib().dg_autotune(self.ctx, C.c_void_p(cost.data_ptr()), int(reps), C.byref(t)), self.ctx)
        return t.as_dict()

    # -- whole steps as CUDA graphs (the context needs a non-default stream)
    def graph_capture(self, cost, refine_spacing_m=0.0, refine_window_m=0.0):
        if cost.dtype != self.dtype or not cost.is_cuda or cost.numel() != self.nrows * self.nlon:
            raise ValueError("cost must be a CUDA tensor of the context's precision and grid size")
        self._keep["graph_cost"] = cost
        with self.torch.cuda.device(self.device):
            _check(lib().dg_graph_capture(self.ctx, C.c_void_p(cost.data_ptr()), float(refine_spacing_m),
                                          float(refine_window_m)), self.ctx)

    def graph_launch(self):
        _check(lib().dg_graph_launch(self.ctx), self.ctx)

    def graph_fix(self):
        f = dg_fix()
        _check(lib().dg_graph_fix(self.ctx, C.byref(f)), self.ctx)
        return f.as_dict()

    def detect(self, cost, threshold, relative=False, radius=3, max_peaks=16):
        if cost.dtype != self.dtype or not cost.is_cuda:
            raise ValueError("cost must be a CUDA tensor of the context's precision")
        return dg_detect(self.ctx, cost.data_ptr(), threshold, relative, radius, max_peaks)

    def sync(self):
        dg_sync(self.ctx)

    # -- inspection
    def grid_ecef(self):
        out = self.torch.empty((3, self.nrows * self.nlon), dtype=self.torch.float64, device=self.device)
        dg_grid_ecef(self.ctx, out.data_ptr())
        return out

    def step_geometry(self, step):
        torch = self.torch
        G = self.nrows * self.nlon
        lag = torch.empty(G, dtype=torch.int32, device=self.device)
        D = torch.empty(G, dtype=torch.float64, device=self.device)
        nu = torch.empty(G, dtype=torch.float64, device=self.device)
        dg_step_geometry(self.ctx, step, lag.data_ptr(), D.data_ptr(), nu.data_ptr())
        return lag, D, nu

    def kernel_time(self, kernel_class):
        return dg_kernel_time(self.ctx, kernel_class)

    def reset_counters(self):
        dg_reset_counters(self.ctx)

    def launch_count(self):
        return dg_launch_count(self.ctx)

    def cdft_work(self):
        return dg_cdft_work(self.ctx)

    def set_grid(self, grid):
        """Move the context to another (whole) grid, keeping its captures."""
        g = grid if isinstance(grid, dg_grid) else dg_grid.from_dict(grid)
        _check(lib().dg_set_grid(self.ctx, C.byref(g)), self.ctx)
        self.grid = {k: getattr(g, k) for k, _ in dg_grid._fields_}
        self.nrows = int(g.nlat)
        self.nlon = int(g.nlon)

    def search_regions(self, regions, refine_spacing_m=0.0, refine_window_m=0.0, costs=None):
        """Cost surfaces of several equal-size regions, then the dense
        re-evaluation around the best one: (fix dict, best index, costs)."""
        torch = self.torch
        arr = (dg_grid * len(regions))(*[g if isinstance(g, dg_grid) else dg_grid.from_dict(g) for g in regions])
        n = len(regions)
        shape = (n, int(arr[0].nlat), int(arr[0].nlon))
        if costs is None:
            costs = torch.empty(shape, dtype=self.dtype, device=self.device)
        if costs.dtype != self.dtype or not costs.is_cuda or not costs.is_contiguous() or costs.numel() < np.prod(shape):
            raise ValueError("costs must be a contiguous CUDA tensor of the context's precision")
        fix, best = dg_fix(), C.c_int32()
        _check(lib().dg_search_regions(self.ctx, arr, n, C.c_void_p(costs.data_ptr()), float(refine_spacing_m),
                                       float(refine_window_m), C.byref(fix), C.byref(best)), self.ctx)
        g = arr[best.value]
        self.grid = {k: getattr(g, k) for k, _ in dg_grid._fields_}
        self.nrows, self.nlon = int(g.nlat), int(g.nlon)
        return fix.as_dict(), best.value, costs

    def coarse_maps(self, bins=0, chunk=0, out=None):
        """Coarse delay-Doppler maps back-projected onto the grid's cells:
        float32 (K, nlat - 1, nlon - 1) on the device (dg_coarse_maps)."""
        torch = self.torch
        shape = (self.K, int(self.grid["nlat"]) - 1, self.nlon - 1)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < np.prod(shape):
            raise ValueError("out must be a contiguous float32 CUDA tensor of K x (nlat-1) x (nlon-1)")
        _check(lib().dg_coarse_maps(self.ctx, int(bins), int(chunk), C.c_void_p(out.data_ptr())), self.ctx)
        return out

    def coarse_inspect(self):
        """(A as float32 (K, C, bins) on the device, per-snapshot parameters
        [dict], (bins, chunk, C)) of the last coarse maps."""
        torch = self.torch
        shape = (C.c_int32 * 3)()
        _check(lib().dg_coarse_inspect(self.ctx, None, None, shape), self.ctx)
        Q, M, cap = shape[0], shape[1], shape[2]
        A = torch.empty((self.K, cap, Q), dtype=torch.float32, device=self.device)
        steps = (dg_coarse_step * self.K)()
        _check(lib().dg_coarse_inspect(self.ctx, C.c_void_p(A.data_ptr()), steps, shape), self.ctx)
        return A, [st.as_dict() for st in steps], (Q, M, cap)

    def cdft_chunks(self):
        """(shortest, longest) chunk the last CDFT surface used."""
        lo, hi = C.c_int32(), C.c_int32()
        _check(lib().dg_cdft_chunks(self.ctx, C.byref(lo), C.byref(hi)), self.ctx)
        return lo.value, hi.value

    def close(self):
        if getattr(self, "ctx", None):
            dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
