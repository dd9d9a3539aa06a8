"""Seeded synthetic inputs for the Chebyshev--Jacobi transform workloads.

This module draws random numbers and nothing else: it holds none of the
transform's arithmetic, so both the CPU oracle (test infrastructure) and the
CUDA path can be fed from it without sharing any method code.

Workload recipes follow the paper's own synthetic experiments (Sec. 5: expansion
coefficients drawn from U(0,1) or U(-1,1) n^-2, Jacobi parameters drawn from
U(-1/2,1/2)) scaled to the shapes this library is measured on:

* ``decaying_coefficients(N, p, seed)``: c_n = g_n / (n+1)^p, g_n ~ N(0,1).
* ``jacobi_parameters(seed)``: (alpha, beta) ~ U[-0.45, 0.45]^2.
* ``batch_workload(count, seed)``: N log-uniform in [64, 65536] (integers, so
  usually not a power of two), per-item (alpha, beta), direction Bernoulli(1/2),
  coefficients N(0,1)/(n+1).

All generators use NumPy's PCG64 with base seed 20261203; item t of a
workload draws from the stream ``seed + t``.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20261203


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _power(x: np.ndarray, p: float) -> np.ndarray:
    """x^p, bit-identical on every platform for the exponents the workloads use: integer and
    half-integer p through products and the correctly rounded square root (a libm pow may
    round differently on different machines), other p through numpy's power."""
    if p == 0:
        return np.ones_like(x)
    k = int(np.floor(p))
    if p == k or p - k == 0.5:
        out = np.ones_like(x)
        for _ in range(k):
            out = out * x
        return out * np.sqrt(x) if p != k else out
    return x ** p


def decaying_coefficients(N: int, p: float, seed: int = BASE_SEED) -> np.ndarray:
    """c_n = g_n/(n+1)^p for n = 0..N with g_n i.i.d. standard normal (float64)."""
    g = rng(seed).standard_normal(N + 1)
    n = np.arange(N + 1, dtype=np.float64)
    return g / _power(n + 1.0, p)


def uniform_coefficients(N: int, seed: int = BASE_SEED) -> np.ndarray:
    """c_n ~ U(0,1): the paper's 'irregular function' coefficients (Fig. 3)."""
    return rng(seed).uniform(0.0, 1.0, N + 1)


def jacobi_parameters(seed: int = BASE_SEED, lo: float = -0.45, hi: float = 0.45):
    """(alpha, beta) drawn uniformly from [lo, hi]^2."""
    r = rng(seed)
    a, b = r.uniform(lo, hi, 2)
    return float(a), float(b)


def single_workload(Ns=(1 << 12, 1 << 14, 1 << 16, 1 << 18), seed: int = BASE_SEED, p: float = 1.5):
    """One item per N: (N, alpha, beta, coefficients) with c_n = g_n/(n+1)^p."""
    items = []
    for t, N in enumerate(Ns):
        a, b = jacobi_parameters(seed + 1000 + t)
        items.append((int(N), a, b, decaying_coefficients(int(N), p, seed + t)))
    return items


def batch_workload(count: int = 4096, seed: int = BASE_SEED, nmin: int = 64, nmax: int = 65536):
    """Uneven batch: list of (N, alpha, beta, direction, coefficients).

    direction is +1 (forward) or -1 (inverse)."""
    r = rng(seed)
    logN = r.uniform(np.log(nmin), np.log(nmax), count)
    Ns = np.clip(np.rint(np.exp(logN)).astype(np.int64), nmin, nmax)
    ab = r.uniform(-0.45, 0.45, (count, 2))
    dirs = np.where(r.uniform(0.0, 1.0, count) < 0.5, 1, -1)
    items = []
    for t in range(count):
        N = int(Ns[t])
        items.append((N, float(ab[t, 0]), float(ab[t, 1]), int(dirs[t]),
                      decaying_coefficients(N, 1.0, seed + 1 + t)))
    return items


def serving_requests(count: int, seed: int = BASE_SEED, nmin: int = 128, nmax: int = 1 << 18):
    """Request stream: N log-uniform in [nmin, nmax], (alpha, beta) ~ U[-0.45, 0.45]^2,
    direction Bernoulli(1/2) (+1 forward, -1 inverse), c_n = g_n/(n+1)."""
    r = rng(seed)
    out = []
    for t in range(count):
        N = int(np.clip(np.rint(np.exp(r.uniform(np.log(nmin), np.log(nmax)))), nmin, nmax))
        a, b = r.uniform(-0.45, 0.45, 2)
        d = 1 if r.uniform() < 0.5 else -1
        out.append((N, float(a), float(b), d, decaying_coefficients(N, 1.0, seed + 7 + t)))
    return out


def mixed_large_workload(count: int = 64, N: int = 1 << 20, seed: int = BASE_SEED):
    """count transforms of degree N, (alpha, beta) ~ U[-0.45, 0.45]^2 each, forward and
    inverse alternating, c_n = g_n/(n+1)."""
    r = rng(seed + 5000)
    out = []
    for t in range(count):
        a, b = r.uniform(-0.45, 0.45, 2)
        out.append((N, float(a), float(b), 1 if t % 2 == 0 else -1, decaying_coefficients(N, 1.0, seed + 6000 + t)))
    return out


def irregular_coefficients(N: int, seed: int = BASE_SEED) -> np.ndarray:
    """c_n ~ U(0,1): coefficients of an irregular function (the paper's Fig. 3, left)."""
    return rng(seed).uniform(0.0, 1.0, N + 1)


def continuous_coefficients(N: int, seed: int = BASE_SEED) -> np.ndarray:
    """c_n ~ U(-1,1) / (n+1)^2: coefficients of a continuous function (the paper's Fig. 3,
    right; (n+1) so that c_0 is finite)."""
    n = np.arange(N + 1, dtype=np.float64)
    return rng(seed).uniform(-1.0, 1.0, N + 1) / _power(n + 1.0, 2)


SHIFTED_PARAMETERS = ((1.5, 0.25), (0.1, 1.3))


def shifted_workload(N: int = 1 << 16, seed: int = BASE_SEED):
    """Transforms with one parameter in (1/2, 3/2] (reached by one integer shift, Sec. 1.2):
    [(N, alpha, beta, c)] for each pair of SHIFTED_PARAMETERS, c_n = g_n/(n+1)^1.5."""
    c = decaying_coefficients(N, 1.5, seed + 77)
    return [(N, a, b, c) for a, b in SHIFTED_PARAMETERS]
