"""The plans' partition (Sec. 2.2), read through cjt_get_partition, equals the paper's
partition evaluated independently in mpmath (tests/golden/partition_ref.json, written by
tests/golden/make_partition.py from oracle/partition.py): n_M, the block ratio alpha_N and
every block (j_k, i_k^1, i_k^2), on the forward grid and on the inverse transform's 2G grid,
for the default grid (2^a, 3 2^a or 5 2^a) and, for N of none of these forms, the power-of-two grid.
A correct but more conservative partition (more recurrence, smaller boxes) fails here."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "partition_ref.json")


@pytest.fixture(scope="module")
def cjt():
    import __graft_entry__ as ge
    ge.build()
    from paper_1602_02618_gb300 import cjt as mod
    assert torch.cuda.is_available()
    return mod


def load():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", range(len(load())))
def test_partition_equals_reference(cjt, case):
    c = load()[case]
    d = cjt.CJT_FWD if c["direction"] == "forward" else cjt.CJT_INV
    plan = cjt.Plan(c["N"], c["alpha"], c["beta"], M=c["M"], directions=d, expansion=cjt.CJT_EXPANSION_HAHN,
                    grid=c["grid"])
    info = plan.info()
    assert info["n_M"] == c["n_M"]
    assert abs(info["ratio"] - c["ratio"]) <= 1e-15 * c["ratio"]
    assert (info["grid_fwd"] if d == cjt.CJT_FWD else info["grid_inv"]) == c["Ng"]
    got = [list(b) for b in cjt.partition(plan, d)]
    assert got == c["blocks"], (got, c["blocks"])
    plan.close()
