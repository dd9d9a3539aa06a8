"""Thin Python binding of the C ABI in include/cjt.h (argument marshalling only).

Every step of a transform runs in the CUDA library ``_build/libcjt.so``;
PyTorch is used only to hold device memory and to name CUDA streams.  If the
library has not been built (``__graft_entry__.build()`` or
``python paper_1602_02618_gb300/build.py``) every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcjt.so")

CJT_OK = 0
CJT_EINVAL = -1
CJT_EDOMAIN = -2
CJT_ENOMEM = -3
CJT_ECUDA = -4
CJT_ETIMEOUT = -5
CJT_EBUSY = -6
CJT_EUNSUPPORTED = -7
CJT_EDIRECTION = -8
CJT_FP64 = 0
CJT_MIXED = 1
CJT_DFLOAT = 2
CJT_FWD = 1
CJT_INV = 2
CJT_EXPANSION_AUTO = 0
CJT_EXPANSION_HAHN = 1
CJT_EXPANSION_ULTRASPHERICAL = 2
CJT_OVERLAP_AUTO = 0
CJT_OVERLAP_ASY_FIRST = 1
CJT_OVERLAP_EQUAL = 2
CJT_OVERLAP_REC_FIRST = 3


class cjt_plan_opts(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("eps", ctypes.c_double), ("precision", ctypes.c_int),
                ("directions", ctypes.c_int), ("ratio", ctypes.c_double), ("seg_len", ctypes.c_int),
                ("use_asy", ctypes.c_int), ("shared_workspace", ctypes.c_int), ("rec_store", ctypes.c_int),
                ("expansion", ctypes.c_int), ("grid", ctypes.c_int), ("overlap", ctypes.c_int),
                ("seg_whole", ctypes.c_int)]


class cjt_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("M", ctypes.c_int), ("precision", ctypes.c_int), ("directions", ctypes.c_int),
                ("n_M", ctypes.c_int64), ("ratio", ctypes.c_double), ("nblk_fwd", ctypes.c_int),
                ("nblk_inv", ctypes.c_int), ("rec_steps_fwd", ctypes.c_int64), ("rec_steps_inv", ctypes.c_int64),
                ("fft_len_fwd", ctypes.c_int64), ("fft_len_inv", ctypes.c_int64), ("nfft_fwd", ctypes.c_int64),
                ("nfft_inv", ctypes.c_int64), ("rec_items_fwd", ctypes.c_int64), ("rec_items_inv", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("plan_ms", ctypes.c_double), ("kernels_fwd", ctypes.c_int64),
                ("kernels_inv", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("rec_store_bytes", ctypes.c_int64), ("shift_alpha", ctypes.c_int), ("shift_beta", ctypes.c_int),
                ("expansion", ctypes.c_int), ("grid_fwd", ctypes.c_int64), ("grid_inv", ctypes.c_int64),
                ("parity_fold", ctypes.c_int), ("overlap", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


EXPORTED = ["cjt_plan_opts_default", "cjt_plan", "cjt_destroy", "cjt_get_info", "cjt_forward", "cjt_inverse",
            "cjt_execute_host", "cjt_execute_batched", "cjt_sync", "cjt_strerror", "cjt_last_cuda_error",
            "cjt_version", "cjt_set_profiling", "cjt_get_profile", "cjt_microbench_fma", "cjt_cheb_coeffs_noalloc",
            "cjt_forward_ws", "cjt_inverse_ws", "cjt_batch_create", "cjt_batch_launch", "cjt_batch_info",
            "cjt_batch_destroy", "cjt_jacobi_to_jacobi", "cjt_asy_coefficient", "cjt_asy_eval",
            "cjt_rec_coefficients", "cjt_error_bound", "cjt_batch_launch_host", "cjt_batch_set_profiling",
            "cjt_batch_get_profile", "cjt_get_partition", "cjt_fft_set_config", "cjt_fft_get_config",
            "cjt_fft_time"]

NOALLOC_MAX_N = 65536

BSTAGES = ["fft_asy", "fft_dct", "rec", "rec_stored", "reduce", "pack", "combine", "other"]

STAGES = ["fwd_rec", "fwd_pack", "fwd_fft", "fwd_combine", "fwd_dct", "inv_front", "inv_pack", "inv_fft",
          "inv_rec", "inv_combine"]

_lock = threading.Lock()
_lib = None


class CJTError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        lib = _lib
        msg = lib.cjt_strerror(code).decode() if lib else str(code)
        extra = lib.cjt_last_cuda_error().decode() if (lib and code == CJT_ECUDA) else ""
        super().__init__("%s failed: %s (%d)%s" % (what, msg, code, (" -- " + extra) if extra else ""))


def load(path: str = LIB_PATH):
    """Load libcjt.so and declare its signatures; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: build it with __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        vp, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.cjt_plan_opts_default.argtypes = [ctypes.POINTER(cjt_plan_opts)]
        lib.cjt_plan.argtypes = [ctypes.POINTER(vp), i64, d, d, ctypes.POINTER(cjt_plan_opts), vp]
        lib.cjt_destroy.argtypes = [vp]
        lib.cjt_destroy.restype = None
        lib.cjt_get_info.argtypes = [vp, ctypes.POINTER(cjt_plan_info)]
        lib.cjt_forward.argtypes = [vp, vp, vp, vp]
        lib.cjt_inverse.argtypes = [vp, vp, vp, vp]
        lib.cjt_execute_host.argtypes = [vp, i, vp, vp, vp]
        lib.cjt_execute_batched.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int8),
                                            ctypes.POINTER(i64), vp, vp, vp]
        lib.cjt_sync.argtypes = [vp]
        lib.cjt_set_profiling.argtypes = [vp, i]
        lib.cjt_get_profile.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64), i]
        lib.cjt_microbench_fma.argtypes = [i, ctypes.POINTER(d), vp]
        lib.cjt_cheb_coeffs_noalloc.argtypes = [i64, vp, vp, vp]
        lib.cjt_forward_ws.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.cjt_inverse_ws.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.cjt_jacobi_to_jacobi.argtypes = [vp, vp, vp, vp, vp]
        lib.cjt_asy_coefficient.argtypes = [d, d, i, i64, i, ctypes.POINTER(d)]
        lib.cjt_asy_eval.argtypes = [d, d, i, i, i64, i64, i64, ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.cjt_rec_coefficients.argtypes = [d, d, i64, ctypes.POINTER(d)]
        lib.cjt_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int8),
                                         ctypes.POINTER(i64), vp, vp, i]
        lib.cjt_batch_launch.argtypes = [vp, vp]
        lib.cjt_batch_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.cjt_batch_destroy.argtypes = [vp]
        lib.cjt_batch_destroy.restype = None
        lib.cjt_batch_launch_host.argtypes = [vp, vp, vp, vp]
        lib.cjt_batch_set_profiling.argtypes = [vp, i]
        lib.cjt_batch_get_profile.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64), i]
        lib.cjt_error_bound.argtypes = [vp, i, ctypes.POINTER(d)]
        lib.cjt_get_partition.argtypes = [vp, i, i, ctypes.POINTER(i64), ctypes.POINTER(i)]
        lib.cjt_fft_set_config.argtypes = [i, i, i, i, i]
        lib.cjt_fft_get_config.argtypes = [i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.cjt_fft_time.argtypes = [i, i, i64, i, ctypes.POINTER(d), vp]
        lib.cjt_strerror.argtypes = [i]
        lib.cjt_strerror.restype = ctypes.c_char_p
        lib.cjt_last_cuda_error.restype = ctypes.c_char_p
        lib.cjt_version.restype = ctypes.c_char_p
        for name in ("cjt_plan_opts_default", "cjt_plan", "cjt_get_info", "cjt_forward", "cjt_inverse",
                     "cjt_execute_host", "cjt_execute_batched", "cjt_sync", "cjt_set_profiling", "cjt_get_profile",
                     "cjt_microbench_fma", "cjt_cheb_coeffs_noalloc", "cjt_forward_ws", "cjt_inverse_ws",
                     "cjt_batch_create", "cjt_batch_launch", "cjt_batch_info", "cjt_jacobi_to_jacobi",
                     "cjt_asy_coefficient", "cjt_asy_eval", "cjt_rec_coefficients", "cjt_error_bound",
                     "cjt_batch_launch_host", "cjt_batch_set_profiling", "cjt_batch_get_profile",
                     "cjt_get_partition", "cjt_fft_set_config", "cjt_fft_get_config", "cjt_fft_time"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def _check(rc, what):
    if rc != CJT_OK:
        raise CJTError(rc, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if t.numel() < n:
        raise ValueError("tensor has %d elements, need %d" % (t.numel(), n))
    # the library launches on the current device, where its plans and arrays live
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError("tensor on cuda:%d while cuda:%d is current; call under torch.cuda.device(%d)"
                         % (t.device.index, cur, t.device.index))
    return ctypes.c_void_p(t.data_ptr())


def _dev_buf(t, what):
    """Pointer of a caller's device scratch tensor (any dtype): contiguous, on the current
    CUDA device, so that the library never receives a host address."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA tensor" % what)
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError("%s on cuda:%d while cuda:%d is current" % (what, t.device.index, cur))
    return ctypes.c_void_p(t.data_ptr()), t.numel() * t.element_size()


def _host_buf(a, n, what, writable=False):
    """Pointer of a host float64 array holding at least n values (C-contiguous)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("%s must be a C-contiguous float64 numpy array" % what)
    if writable and not a.flags.writeable:
        raise ValueError("%s is read-only" % what)
    if a.size < n:
        raise ValueError("%s has %d values, need %d" % (what, a.size, n))
    return ctypes.c_void_p(a.ctypes.data)


def default_opts() -> cjt_plan_opts:
    o = cjt_plan_opts()
    _check(load().cjt_plan_opts_default(ctypes.byref(o)), "cjt_plan_opts_default")
    return o


class Plan:
    """A cjt_plan_t: device-resident tables for degree N and parameters (alpha, beta)."""

    def __init__(self, N: int, alpha: float, beta: float, M: int = 0, eps: float = 0.0, precision: int = CJT_FP64,
                 directions: int = 0, ratio: float = 0.0, seg_len: int = 0, use_asy: int = 0,
                 shared_workspace: bool = False, rec_store: int = 0, expansion: int = CJT_EXPANSION_AUTO,
                 grid: int = 0, overlap: int = CJT_OVERLAP_AUTO, seg_whole: int = 0, stream=None):
        lib = load()
        o = cjt_plan_opts(M, eps, precision, directions, ratio, seg_len, use_asy, 1 if shared_workspace else 0,
                          int(rec_store), int(expansion), int(grid), int(overlap), int(seg_whole))
        h = ctypes.c_void_p()
        _check(lib.cjt_plan(ctypes.byref(h), int(N), float(alpha), float(beta), ctypes.byref(o),
                            _stream_handle(stream)), "cjt_plan")
        self._h = h
        self.N = int(N)
        self.alpha = float(alpha)
        self.beta = float(beta)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = cjt_plan_info()
        _check(load().cjt_get_info(self._h, ctypes.byref(inf)), "cjt_get_info")
        return inf.as_dict()

    def set_profiling(self, on: bool = True):
        _check(load().cjt_set_profiling(self._h, 1 if on else 0), "cjt_set_profiling")

    def profile(self):
        """{stage: (total ms, launches)} of the executions since the last call."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(load().cjt_get_profile(self._h, ms, cnt, n), "cjt_get_profile")
        return {STAGES[s]: (ms[s], cnt[s]) for s in range(n)}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().cjt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cjt_forward(plan: Plan, c_jac, c_cheb=None, stream=None):
    """c_cheb = T_N^{-1} P_N c_jac on the device (float64 CUDA tensors of N+1 values)."""
    import torch
    n = plan.N + 1
    if c_cheb is None:
        c_cheb = torch.empty(n, dtype=torch.float64, device=c_jac.device)
    _check(load().cjt_forward(plan.handle, _dev_ptr(c_jac, n), _dev_ptr(c_cheb, n), _stream_handle(stream)),
           "cjt_forward")
    return c_cheb


def cjt_inverse(plan: Plan, c_cheb, c_jac=None, stream=None):
    """c_jac = P_N^{-1} T_N c_cheb on the device."""
    import torch
    n = plan.N + 1
    if c_jac is None:
        c_jac = torch.empty(n, dtype=torch.float64, device=c_cheb.device)
    _check(load().cjt_inverse(plan.handle, _dev_ptr(c_cheb, n), _dev_ptr(c_jac, n), _stream_handle(stream)),
           "cjt_inverse")
    return c_jac


def cjt_execute_host(plan: Plan, direction: int, x: np.ndarray, out: np.ndarray = None, stream=None):
    """Host-to-host transform through the library's own staging buffers (synchronous)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.size != plan.N + 1:
        raise ValueError("expected %d values" % (plan.N + 1))
    if out is None:
        out = np.empty_like(x)
    po = _host_buf(out, plan.N + 1, "out", writable=True)
    _check(load().cjt_execute_host(plan.handle, int(direction), _host_buf(x, plan.N + 1, "x"), po,
                                   _stream_handle(stream)), "cjt_execute_host")
    return out


def cjt_execute_batched(plans, dirs, offsets, x_dev, out_dev, stream=None):
    """Items t: plans[t] in direction dirs[t] on x_dev[offsets[t]:] -> out_dev[offsets[t]:]."""
    count = len(plans)
    arr = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
    d = (ctypes.c_int8 * count)(*[int(v) for v in dirs])
    off = (ctypes.c_int64 * count)(*[int(v) for v in offsets])
    total = max((int(o) + p.N + 1 for o, p in zip(offsets, plans)), default=0)
    _check(load().cjt_execute_batched(count, arr, d, off, _dev_ptr(x_dev, total), _dev_ptr(out_dev, total),
                                      _stream_handle(stream)), "cjt_execute_batched")
    return out_dev


def cjt_jacobi_to_jacobi(plan_from: Plan, plan_to: Plan, c_in, c_out=None, stream=None):
    """Coefficients in the Jacobi basis of plan_to of the expansion c_in in the basis of
    plan_from (forward of plan_from, then inverse of plan_to, on the device)."""
    import torch
    n = plan_from.N + 1
    if c_out is None:
        c_out = torch.empty(n, dtype=torch.float64, device=c_in.device)
    _check(load().cjt_jacobi_to_jacobi(plan_from.handle, plan_to.handle, _dev_ptr(c_in, n), _dev_ptr(c_out, n),
                                       _stream_handle(stream)), "cjt_jacobi_to_jacobi")
    return c_out


def cjt_forward_ws(plan: Plan, c_jac, c_cheb, workspace, stream=None):
    """Forward transform borrowing `workspace` (a CUDA tensor of >= workspace_bytes bytes)."""
    n = plan.N + 1
    ws, nbytes = _dev_buf(workspace, "workspace")
    _check(load().cjt_forward_ws(plan.handle, _dev_ptr(c_jac, n), _dev_ptr(c_cheb, n), ws, nbytes,
                                 _stream_handle(stream)), "cjt_forward_ws")
    return c_cheb


def cjt_inverse_ws(plan: Plan, c_cheb, c_jac, workspace, stream=None):
    """Inverse transform borrowing `workspace` (a CUDA tensor of >= workspace_bytes bytes)."""
    n = plan.N + 1
    ws, nbytes = _dev_buf(workspace, "workspace")
    _check(load().cjt_inverse_ws(plan.handle, _dev_ptr(c_cheb, n), _dev_ptr(c_jac, n), ws, nbytes,
                                 _stream_handle(stream)), "cjt_inverse_ws")
    return c_jac


def fft_set_config(precision: int, log2L: int, ctas_per_sm: int = 4, split: int = 0, single_max_log2: int = 12):
    """Launch configuration of the transforms of one (precision, length) class (process-wide)."""
    _check(load().cjt_fft_set_config(int(precision), int(log2L), int(ctas_per_sm), int(split), int(single_max_log2)),
           "cjt_fft_set_config")


def fft_get_config(precision: int, log2L: int):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().cjt_fft_get_config(int(precision), int(log2L), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "cjt_fft_get_config")
    return {"ctas_per_sm": a.value, "split": b.value, "single_max_log2": c.value}


def fft_time(precision: int, log2L: int, batch: int, reps: int = 3, stream=None) -> float:
    """Milliseconds of `batch` transforms of length 2^log2L under the current configuration."""
    v = ctypes.c_double()
    _check(load().cjt_fft_time(int(precision), int(log2L), int(batch), int(reps), ctypes.byref(v),
                               _stream_handle(stream)), "cjt_fft_time")
    return v.value


def partition(plan: Plan, direction: int):
    """The plan's blocks on the grid of `direction`: a list of (j_k, i_k^1, i_k^2), outermost
    first (Sec. 2.2)."""
    cap = 64
    boxes = (ctypes.c_int64 * (3 * cap))()
    n = ctypes.c_int()
    _check(load().cjt_get_partition(plan.handle, int(direction), cap, boxes, ctypes.byref(n)), "cjt_get_partition")
    return [(boxes[3 * k], boxes[3 * k + 1], boxes[3 * k + 2]) for k in range(n.value)]


def error_bound(plan: Plan, direction: int) -> float:
    """Stated error bound of the plan's transform in `direction`, per unit ||c_in||_1."""
    v = ctypes.c_double()
    _check(load().cjt_error_bound(plan.handle, int(direction), ctypes.byref(v)), "cjt_error_bound")
    return v.value


class Batch:
    """cjt_batch_t: a batched execution captured into one CUDA graph."""

    def __init__(self, plans, dirs, offsets, x_dev, out_dev, nstreams: int = 0):
        count = len(plans)
        arr = (ctypes.c_void_p * count)(*[p.handle.value for p in plans])
        d = (ctypes.c_int8 * count)(*[int(v) for v in dirs])
        off = (ctypes.c_int64 * count)(*[int(v) for v in offsets])
        total = max(int(o) + p.N + 1 for o, p in zip(offsets, plans))
        h = ctypes.c_void_p()
        _check(load().cjt_batch_create(ctypes.byref(h), count, arr, d, off, _dev_ptr(x_dev, total),
                                       _dev_ptr(out_dev, total), int(nstreams)), "cjt_batch_create")
        self._h = h
        self._keep = (plans, x_dev, out_dev)
        self.total = total

    def launch(self, stream=None):
        _check(load().cjt_batch_launch(self._h, _stream_handle(stream)), "cjt_batch_launch")

    def launch_host(self, x_host: np.ndarray, out_host: np.ndarray, stream=None):
        """Host input -> device -> replay -> host output, synchronous (whole-batch arrays of
        at least max_t (offsets[t] + N_t + 1) values)."""
        px = _host_buf(x_host, self.total, "x_host")
        po = _host_buf(out_host, self.total, "out_host", writable=True)
        _check(load().cjt_batch_launch_host(self._h, px, po, _stream_handle(stream)), "cjt_batch_launch_host")
        return out_host

    def set_profiling(self, on: bool = True):
        _check(load().cjt_batch_set_profiling(self._h, 1 if on else 0), "cjt_batch_set_profiling")

    def profile(self):
        """{stage kind: (total ms, launches)} of the profiled launches since the last call."""
        n = len(BSTAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(load().cjt_batch_get_profile(self._h, ms, cnt, n), "cjt_batch_get_profile")
        return {BSTAGES[s]: (ms[s], cnt[s]) for s in range(n)}

    def info(self):
        k, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().cjt_batch_info(self._h, ctypes.byref(k), ctypes.byref(b)), "cjt_batch_info")
        return {"kernels": k.value, "arena_bytes": b.value}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().cjt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cjt_sync(stream=None):
    _check(load().cjt_sync(_stream_handle(stream)), "cjt_sync")


def cjt_cheb_coeffs_noalloc(values, c_cheb, stream=None):
    """Chebyshev coefficients from values at the N+1 Lobatto points through the
    allocation-free entry point (working memory in a fixed device array; both
    tensors must already exist, N = values.numel() - 1 a power of two <= 65536)."""
    n = values.numel()
    _check(load().cjt_cheb_coeffs_noalloc(n - 1, _dev_ptr(values, n), _dev_ptr(c_cheb, n), _stream_handle(stream)),
           "cjt_cheb_coeffs_noalloc")
    return c_cheb


def microbench_fma(kind=True, stream=None) -> float:
    """Measured dependent multiply-add throughput of the device in FLOP/s: kind True/1 FP64,
    False/0 FP32, 2 double-float."""
    v = ctypes.c_double()
    _check(load().cjt_microbench_fma(int(kind), ctypes.byref(v), _stream_handle(stream)),
           "cjt_microbench_fma")
    return v.value


def asy_coefficient(alpha: float, beta: float, n: int, m: int, expansion: int = CJT_EXPANSION_AUTO) -> float:
    """C_{n,m} of the expansion a plan for (alpha, beta) uses (host only, no GPU)."""
    C = ctypes.c_double()
    _check(load().cjt_asy_coefficient(float(alpha), float(beta), int(expansion), int(n), int(m), ctypes.byref(C)),
           "cjt_asy_coefficient")
    return C.value


def asy_eval(alpha: float, beta: float, M: int, n: int, i: int, Ng: int, expansion: int = CJT_EXPANSION_AUTO):
    """(value, bound): the plan's M-term expansion of P_n(cos(pi i / Ng)) and the bound on
    its remainder that the partition uses (host only, no GPU)."""
    v, b = ctypes.c_double(), ctypes.c_double()
    _check(load().cjt_asy_eval(float(alpha), float(beta), int(expansion), int(M), int(n), int(i), int(Ng),
                               ctypes.byref(v), ctypes.byref(b)), "cjt_asy_eval")
    return v.value, b.value


REC_FIELDS = ("A", "B", "C", "rf_p", "rf_m", "rb_p", "rb_m", "Ce_p", "Ce_m", "Cr_p", "Cr_m")


def rec_coefficients(alpha: float, beta: float, n: int) -> dict:
    """The plan's recurrence-table entries for degree n (host only, no GPU): A_n, B_n, C_n,
    the Reinsch ratios r^f_n(+-1), r^b_n(+-1), C_n / r^f_{n-1}(+-1) and C_n r^b_n(+-1)."""
    out = (ctypes.c_double * len(REC_FIELDS))()
    _check(load().cjt_rec_coefficients(float(alpha), float(beta), int(n), out), "cjt_rec_coefficients")
    return dict(zip(REC_FIELDS, list(out)))


def version() -> str:
    return load().cjt_version().decode()
