"""The stored full-size oracle outputs (tests/golden/oracle_*.npz, written by
tests/golden/make_fullsize.py from the CPU oracle) are pinned here against what the
mathematics fixes, independently of how they were computed:

  * each fixture's input is the seeded workload item it names (digest of the regenerated
    coefficients, N, alpha, beta, direction);
  * forward fixtures (all entries): sum_k c_k T_k(x_j) = sum_n c_n P_n(x_j) at sampled
    Lobatto points (Eq. "CJT": T_N c_cheb = P_N c_jac), both sides evaluated by the oracle's
    double-double series in O(N) per point;
  * inverse fixtures (all entries): sum_n c_jac_n P_n(x_j) = sum_k c_k T_k(x_j) at sampled
    interior points within the rounding of the stored doubles carried by |P_n(x_j)|, and
    the exact first coefficient c_jac_0 = sum_k c_k mu_k / mu_0 (Eq. "cjintdefn" at n = 0);
  * sampled fixtures (N = 2^20): indices sorted, in range, both ends kept; the plain-double
    inverse's measured error is far below the mixed form's bound it serves.
"""
import hashlib
import os

import numpy as np
import pytest

from paper_1602_02618_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SINGLE = [1 << 12, 1 << 14, 1 << 16, 1 << 18]


def load(name):
    path = os.path.join(GOLDEN, "oracle_%s.npz" % name)
    if not os.path.exists(path):
        pytest.fail("missing oracle fixture %s (run tests/golden/make_fullsize.py)" % path)
    return np.load(path)


def single(N):
    for n, a, b, c in inputs.single_workload(Ns=tuple(SINGLE), seed=inputs.BASE_SEED):
        if n == N:
            return a, b, c
    raise KeyError(N)


def digest(c):
    return hashlib.sha256(np.ascontiguousarray(c, dtype=np.float64).tobytes()).hexdigest()


@pytest.mark.parametrize("N", SINGLE)
def test_forward_fixture(orc, N):
    fx = load("fwd_N%d" % N)
    a, b, c = single(N)
    assert str(fx["input_sha256"]) == digest(c) and int(fx["N"]) == N and int(fx["direction"]) == 1
    assert float(fx["alpha"]) == a and float(fx["beta"]) == b and fx["idx"].size == 0
    out = fx["out"]
    assert out.shape == (N + 1,)
    j = np.unique(np.concatenate([[0, 1, N // 2, N - 1, N], inputs.rng(N + 11).integers(0, N + 1, 24)]))
    lhs = orc.cheb_series(out, j, N)
    rhs = orc.jacobi_series(c, a, b, j, N)
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * (np.abs(out).sum() + np.abs(c).sum())


@pytest.mark.parametrize("N", SINGLE)
def test_inverse_fixture(orc, N):
    fx = load("inv_N%d" % N)
    a, b, c = single(N)
    assert str(fx["input_sha256"]) == digest(c) and int(fx["N"]) == N and int(fx["direction"]) == -1
    out = fx["out"]
    assert out.shape == (N + 1,)
    mu = orc.moments(N, a, b)
    assert abs(out[0] - np.dot(c, mu) / mu[0]) <= 1e-15 * np.abs(c).sum()
    for j in inputs.rng(N + 13).integers(N // 8, 7 * N // 8, 6):
        lhs = orc.jacobi_series(out, a, b, [int(j)], N)[0]
        rhs = orc.cheb_series(c, [int(j)], N)[0]
        P = orc.jacobi_values(N, a, b, int(j), N)
        assert abs(lhs - rhs) <= 4e-16 * float(np.abs(out * P).sum()) + 1e-15 * np.abs(c).sum()


@pytest.mark.parametrize("t", [0, 1])
def test_shifted_inverse_fixture(orc, t):
    """Inverse at N = 2^16 with one parameter in (1/2, 3/2]: the same identities."""
    N, a, b, c = inputs.shifted_workload()[t]
    fx = load("shift%d_inv_N%d" % (t, N))
    assert str(fx["input_sha256"]) == digest(c) and int(fx["N"]) == N and int(fx["direction"]) == -1
    assert float(fx["alpha"]) == a and float(fx["beta"]) == b and fx["idx"].size == 0
    out = fx["out"]
    assert out.shape == (N + 1,)
    mu = orc.moments(N, a, b)
    assert abs(out[0] - np.dot(c, mu) / mu[0]) <= 1e-15 * np.abs(c).sum()
    for j in inputs.rng(N + 17 + t).integers(N // 8, 7 * N // 8, 6):
        lhs = orc.jacobi_series(out, a, b, [int(j)], N)[0]
        rhs = orc.cheb_series(c, [int(j)], N)[0]
        P = orc.jacobi_values(N, a, b, int(j), N)
        assert abs(lhs - rhs) <= 4e-16 * float(np.abs(out * P).sum()) + 1e-15 * np.abs(c).sum()


@pytest.mark.parametrize("name", ["fwd_N1048576", "inv_N1048576"])
def test_sampled_fixtures(name):
    fx = load(name)
    N = int(fx["N"])
    t = 0 if name.startswith("fwd") else 1
    n, a, b, d, c = inputs.mixed_large_workload(2, 1 << 20, seed=inputs.BASE_SEED)[t]
    assert N == n and str(fx["input_sha256"]) == digest(c) and int(fx["direction"]) == d
    idx = fx["idx"]
    assert idx.size == fx["out"].size == 8192 and np.all(np.diff(idx) > 0)
    assert idx[0] == 0 and idx[-1] == N and np.all(np.isfinite(fx["out"]))
    if t == 1:
        assert str(fx["oracle"]) == "plain double"
        assert float(fx["f64_err_N65536"]) < 1e-9
