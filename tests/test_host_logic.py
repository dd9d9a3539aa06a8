"""Host-side logic that needs no GPU: the seeded workload generators and the
autotuner's candidate set and cache file."""
import json

import numpy as np
import pytest

from paper_1602_02618_gb300 import autotune, inputs


def test_batch_workload_shape_and_determinism():
    a = inputs.batch_workload(256)
    b = inputs.batch_workload(256)
    assert len(a) == 256
    Ns = np.array([it[0] for it in a])
    assert Ns.min() >= 64 and Ns.max() <= 65536
    # log-uniform: about half the items lie below the geometric midpoint 2048
    assert 0.35 < np.mean(Ns < 2048) < 0.65
    assert np.mean((Ns & (Ns - 1)) != 0) > 0.9          # mostly not powers of two
    dirs = np.array([it[3] for it in a])
    assert set(dirs) == {1, -1} and 0.35 < np.mean(dirs == 1) < 0.65
    for (N, al, be, d, c), (N2, al2, be2, d2, c2) in zip(a, b):
        assert (N, al, be, d) == (N2, al2, be2, d2) and np.array_equal(c, c2)
        assert -0.45 <= al <= 0.45 and -0.45 <= be <= 0.45
        assert c.shape == (N + 1,) and c.dtype == np.float64
    c = inputs.batch_workload(256, seed=inputs.BASE_SEED + 1)
    assert [it[0] for it in c] != [it[0] for it in a]


def test_coefficient_recipes():
    N = 4096
    g = inputs.rng(inputs.BASE_SEED).standard_normal(N + 1)
    c = inputs.decaying_coefficients(N, 1.5, inputs.BASE_SEED)
    n1 = np.arange(N + 1) + 1.0
    # (n+1)^1.5 as a product with the correctly rounded square root: the same bits on every
    # platform, and within an ulp or two of the power
    assert np.array_equal(c, g / (n1 * np.sqrt(n1)))
    assert np.max(np.abs(c - g / n1 ** 1.5) / np.abs(c)) < 1e-15
    assert np.array_equal(inputs.decaying_coefficients(N, 1.0, 7), inputs.rng(7).standard_normal(N + 1) / n1)
    u = inputs.irregular_coefficients(N)
    assert u.min() >= 0.0 and u.max() < 1.0
    v = inputs.continuous_coefficients(N)
    assert np.all(np.abs(v) <= 1.0 / (np.arange(N + 1) + 1.0) ** 2)
    items = inputs.single_workload()
    assert [it[0] for it in items] == [1 << 12, 1 << 14, 1 << 16, 1 << 18]
    big = inputs.mixed_large_workload(4, 1024)
    assert [it[3] for it in big] == [1, -1, 1, -1] and all(it[0] == 1024 for it in big)
    reqs = inputs.serving_requests(64)
    assert all(128 <= r[0] <= 1 << 18 and r[3] in (1, -1) for r in reqs)


def test_autotune_candidates():
    small = autotune.candidates(1000, 40e9)
    big = autotune.candidates(1 << 20, 40e9)
    for opts in small + big:
        assert opts["M"] >= 5 and opts["seg_len"] in (256, 1024) and opts["rec_store"] in (0, 1)
    # the recurrence-only candidate only when its stored matrix fits the cap
    assert any(o.get("use_asy") == -1 for o in small)
    assert not any(o.get("use_asy") == -1 for o in big)
    assert any(o["rec_store"] == 0 for o in big) and any(o.get("ratio") == 0.05 for o in big)
    assert len({json.dumps(o, sort_keys=True) for o in big}) == len(big)


def test_autotune_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("CJT_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}
    entry = {"k": {"options": {"M": 10, "seg_len": 256, "rec_store": 1}, "ms": 1.5}}
    autotune._save(entry)
    assert autotune._load() == entry
    path.write_text("{not json")
    assert autotune._load() == {}
    # small N never times anything
    assert autotune.best_options(100, 0.1, -0.3) == {"M": 7, "seg_len": 256}
