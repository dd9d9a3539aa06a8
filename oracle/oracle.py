"""Python access to the CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain, slow, double-double C implementation of the paper's
definitions (see cjt_oracle.c for the citations).  Only the test-suite, the
smoke check and the benchmark's CPU-baseline leg and reference arm may import
this module; the library itself never does.

``build()`` compiles ``cjt_oracle.c`` with gcc (OpenMP, -ffp-contract=off so
that the error-free transformations are not contracted into fused
multiply-adds) into ``oracle/_build/libcjt_oracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cjt_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcjt_oracle.so")

_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", "-D_DEFAULT_SOURCE", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            i64, d, i = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            lib.orc_cospi_frac.argtypes = [i64, i64, _dp, _dp]
            lib.orc_rec_coeffs.argtypes = [i64, d, d, _dp, _dp, _dp]
            lib.orc_jacobi_values.argtypes = [i64, d, d, i64, i64, _dp]
            lib.orc_jacobi_series.argtypes = [i64, d, d, _dp, i64, _ip, i64, _dp, _dp, i]
            lib.orc_cheb_series.argtypes = [i64, _dp, i64, _ip, i64, _dp, _dp, i]
            lib.orc_forward.argtypes = [i64, d, d, _dp, _dp, i]
            lib.orc_forward_values.argtypes = [i64, d, d, _dp, _dp, _dp, i]
            lib.orc_forward_f64.argtypes = [i64, d, d, _dp, _dp, i]
            lib.orc_moments.argtypes = [i64, d, d, _dp]
            lib.orc_cc_weights.argtypes = [i64, d, d, _dp, i]
            lib.orc_norm_consts.argtypes = [i64, d, d, _dp]
            lib.orc_inverse.argtypes = [i64, d, d, _dp, _dp, i]
            lib.orc_inverse_f64.argtypes = [i64, d, d, _dp, _dp, i]
            for name in ("orc_jacobi_values", "orc_jacobi_series", "orc_cheb_series", "orc_forward",
                         "orc_forward_values", "orc_forward_f64", "orc_moments", "orc_cc_weights",
                         "orc_norm_consts", "orc_inverse", "orc_inverse_f64"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def cospi_frac(p: int, q: int):
    """cos(pi p/q) as a double-double (hi, lo)."""
    hi, lo = ctypes.c_double(), ctypes.c_double()
    _load().orc_cospi_frac(p, q, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def rec_coeffs(n: int, alpha: float, beta: float):
    A, B, C = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_rec_coeffs(n, alpha, beta, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C))
    return A.value, B.value, C.value


def jacobi_values(nmax: int, alpha: float, beta: float, j: int, grid_N: int) -> np.ndarray:
    """P_n(cos(pi j/grid_N)) for n = 0..nmax."""
    out = np.empty(nmax + 1)
    _check(_load().orc_jacobi_values(nmax, alpha, beta, j, grid_N, _p(out)), "jacobi_values")
    return out


def jacobi_series(c, alpha: float, beta: float, j, grid_N: int, nthreads: int = 0, lo: bool = False):
    """sum_n c_n P_n(cos(pi j/grid_N)) for each j in the index list."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    hi = np.empty(j.size)
    lo_arr = np.empty(j.size)
    _check(_load().orc_jacobi_series(c.size - 1, alpha, beta, _p(c), j.size, j.ctypes.data_as(_ip), grid_N,
                                      _p(hi), _p(lo_arr), nthreads), "jacobi_series")
    return (hi, lo_arr) if lo else hi


def cheb_series(c, j, grid_N: int, nthreads: int = 0, lo: bool = False):
    """sum_k c_k T_k(cos(pi j/grid_N)) for each j in the index list."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    hi = np.empty(j.size)
    lo_arr = np.empty(j.size)
    _check(_load().orc_cheb_series(c.size - 1, _p(c), j.size, j.ctypes.data_as(_ip), grid_N, _p(hi), _p(lo_arr),
                                   nthreads), "cheb_series")
    return (hi, lo_arr) if lo else hi


def forward(c_jac, alpha: float, beta: float, nthreads: int = 0) -> np.ndarray:
    """c_cheb = T_N^{-1} P_N c_jac (double-double internally)."""
    c = np.ascontiguousarray(c_jac, dtype=np.float64)
    out = np.empty_like(c)
    _check(_load().orc_forward(c.size - 1, alpha, beta, _p(c), _p(out), nthreads), "forward")
    return out


def forward_values(c_jac, alpha: float, beta: float, nthreads: int = 0):
    """(hi, lo) of y_j = sum_n c_n P_n(x_j) on the N+1 Lobatto points."""
    c = np.ascontiguousarray(c_jac, dtype=np.float64)
    hi, lo = np.empty_like(c), np.empty_like(c)
    _check(_load().orc_forward_values(c.size - 1, alpha, beta, _p(c), _p(hi), _p(lo), nthreads), "forward_values")
    return hi, lo


def forward_f64(c_jac, alpha: float, beta: float, nthreads: int = 0) -> np.ndarray:
    """Plain-double O(N^2) forward transform (the timed naive baseline)."""
    c = np.ascontiguousarray(c_jac, dtype=np.float64)
    out = np.empty_like(c)
    _check(_load().orc_forward_f64(c.size - 1, alpha, beta, _p(c), _p(out), nthreads), "forward_f64")
    return out


def moments(K: int, alpha: float, beta: float) -> np.ndarray:
    out = np.empty(K + 1)
    _check(_load().orc_moments(K, alpha, beta, _p(out)), "moments")
    return out


def cc_weights(Ng: int, alpha: float, beta: float, nthreads: int = 0) -> np.ndarray:
    out = np.empty(Ng + 1)
    _check(_load().orc_cc_weights(Ng, alpha, beta, _p(out), nthreads), "cc_weights")
    return out


def norm_consts(N: int, alpha: float, beta: float) -> np.ndarray:
    out = np.empty(N + 1)
    _check(_load().orc_norm_consts(N, alpha, beta, _p(out)), "norm_consts")
    return out


def inverse(c_cheb, alpha: float, beta: float, nthreads: int = 0) -> np.ndarray:
    """c_jac = P_N^{-1} T_N c_cheb via the Clenshaw--Curtis quadrature definition."""
    c = np.ascontiguousarray(c_cheb, dtype=np.float64)
    out = np.empty_like(c)
    _check(_load().orc_inverse(c.size - 1, alpha, beta, _p(c), _p(out), nthreads), "inverse")
    return out


def inverse_f64(c_cheb, alpha: float, beta: float, nthreads: int = 0) -> np.ndarray:
    """Plain-double O(N^2) inverse transform (the timed naive baseline)."""
    c = np.ascontiguousarray(c_cheb, dtype=np.float64)
    out = np.empty_like(c)
    _check(_load().orc_inverse_f64(c.size - 1, alpha, beta, _p(c), _p(out), nthreads), "inverse_f64")
    return out


def jacobi_to_jacobi(c, alpha: float, beta: float, gamma: float, delta: float, nthreads: int = 0) -> np.ndarray:
    """Coefficients in P^{(gamma,delta)} of sum_n c_n P_n^{(alpha,beta)}: the forward transform
    of (alpha, beta) followed by the inverse transform of (gamma, delta) (Sec. 5, composition
    of the two transforms)."""
    return inverse(forward(c, alpha, beta, nthreads), gamma, delta, nthreads)
