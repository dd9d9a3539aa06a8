"""Pins of the mpmath partition oracle (oracle/partition.py, Sec. 2.2) and of its stored values
(tests/golden/partition_ref.json):

  * the boxes satisfy their definition: the remainder bound 2 C_{j_k,M} g_M(theta_i) is below
    eps at both end rows and above it just outside (or the row is an end of the grid);
  * the boxes are nested (degrees decrease, rows shrink) and j_k = floor(alpha_N^k Ng) with
    alpha_N = min(1/log(Ng/n_M), 1/2) and n_M from the envelope at pi/2;
  * C_{n,m} of Eq. "Cnmab" satisfies the recurrence in m of Eq. "Cnmabrec" and, at a = b = 0,
    the closed form through the central binomial coefficient;
  * independently computed probe values of the partition (N = 1024 and 2^14, (0.1, -0.3),
    M = 7; two blocks at N = 2^18, M = 13) are reproduced: a cross-check, not the pin.
"""
import json
import math
import os

import pytest

mp = pytest.importorskip("mpmath")

from oracle import partition as P  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "partition_ref.json")


def cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def test_hahn_C_recurrence_and_closed_form():
    for n in (3, 17, 200):
        for m in (1, 4, 9):
            for a, b in ((0.1, -0.3), (0.45, 0.45), (-0.5, 0.5)):
                with mp.workdps(P.DPS):
                    lhs = P.hahn_C(n, m, a, b)
                    rhs = P.hahn_C(n, m - 1, a, b) / (2 * (2 * n + mp.mpf(a) + mp.mpf(b) + m + 1))
                    assert abs(lhs - rhs) <= 1e-30 * abs(rhs)
    # a = b = 0, m = 0: C_{n,0} = 2^(2n+1) B(n+1, n+1) / pi = 2^(2n+1) / ((2n+1) pi binom(2n, n))
    for n in (0, 5, 40):
        with mp.workdps(P.DPS):
            want = mp.mpf(2) ** (2 * n + 1) / ((2 * n + 1) * mp.pi * math.comb(2 * n, n))
            assert abs(P.hahn_C(n, 0, 0.0, 0.0) - want) <= 1e-32 * want


@pytest.mark.parametrize("case", range(12))
def test_boxes_satisfy_their_definition(case):
    c = cases()[case]
    Ng, M, a, b, N = c["Ng"], c["M"], c["alpha"], c["beta"], c["N"]
    assert c["n_M"] == P.n_M(M, a, b)
    r = min(1.0 / math.log(Ng / c["n_M"]), 0.5)
    assert c["ratio"] == r
    prev = None
    for k, (j, i1, i2) in enumerate(c["blocks"], start=1):
        assert j == int(mp.floor(mp.mpf(r) ** k * Ng)) and c["n_M"] < j <= N
        assert P.criterion_margin(j, i1, Ng, M, a, b) > 0 and P.criterion_margin(j, i2, Ng, M, a, b) > 0
        assert i1 == 1 or P.criterion_margin(j, i1 - 1, Ng, M, a, b) <= 0
        assert i2 == Ng - 1 or P.criterion_margin(j, i2 + 1, Ng, M, a, b) <= 0
        mid = (i1 + i2) // 2
        assert P.criterion_margin(j, mid, Ng, M, a, b) > 0
        if prev:
            assert j < prev[0] and i1 >= prev[1] and i2 <= prev[2]
        prev = (j, i1, i2)


def test_independent_probe_values():
    got = {(c["N"], c["direction"], c["M"]): (c["n_M"], c["blocks"]) for c in cases()}
    assert got[(1024, "forward", 7)] == (106, [[451, 103, 937], [199, 235, 817]])
    assert got[(16384, "forward", 7)] == (106, [[3250, 235, 16206], [644, 1159, 15424], [127, 6057, 10909]])
    assert got[(262144, "forward", 13)][1][0] == [27930, 98, 262069]
    assert got[(262144, "forward", 13)][1][-1] == [33, 72872, 193739]
