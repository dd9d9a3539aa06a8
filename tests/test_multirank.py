"""The multi-GPU form's host logic on CPU: two ranks over gloo, no GPU.

Transforms are independent, so under torchrun every rank runs its own seeded
shard and the ranks exchange nothing on the data path; the host takes the
slowest rank's time and the sum of the units.  These tests run that logic with
world size 2 on the gloo backend:

* the helpers of paper_1602_02618_gb300.multirank (max and sum over ranks,
  barrier, the job rate) across two processes;
* the shards bench.py builds: rank 0's is the one-GPU workload, rank 1's has
  the same shape and different draws;
* bench.py --impl reference under torchrun: rank 0 alone prints one line.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_seeds_and_env(monkeypatch):
    from paper_1602_02618_gb300 import inputs, multirank
    assert multirank.rank_seed(inputs.BASE_SEED, 0) == inputs.BASE_SEED
    seeds = [multirank.rank_seed(inputs.BASE_SEED, r) for r in range(8)]
    # item t of a workload draws from seed + t with t < 2^20: rank streams never meet
    assert min(np.diff(seeds)) >= 1 << 20
    with pytest.raises(ValueError):
        multirank.rank_seed(inputs.BASE_SEED, -1)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert multirank.env() == (1, 0, 0)
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert multirank.env() == (4, 3, 1)
    monkeypatch.setenv("RANK", "4")
    with pytest.raises(ValueError):
        multirank.env()
    assert multirank.max_over_ranks(2.5) == 2.5 and multirank.sum_over_ranks(2.5) == 2.5
    assert multirank.job_rate(10.0, 4.0) == 2.5
    with pytest.raises(ValueError):
        multirank.job_rate(1.0, 0.0)


WORKER = textwrap.dedent("""
    import json, sys, time
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch.distributed as dist
    from paper_1602_02618_gb300 import inputs, multirank
    import bench

    world, rank, local = multirank.env()
    dist.init_process_group("gloo", init_method="env://")
    mx = multirank.max_over_ranks(rank + 1.5, dist)
    sm = multirank.sum_over_ranks(rank + 1.0, dist)
    # a timed region as bench.py brackets it: barrier, work of unequal length, barrier,
    # the slowest rank's time and the units of all ranks
    items = bench.workload(rank)
    batch = inputs.batch_workload(8, seed=multirank.rank_seed(inputs.BASE_SEED, rank))
    multirank.barrier(dist)
    t0 = time.perf_counter()
    time.sleep(0.05 * (rank + 1))
    mine = time.perf_counter() - t0
    multirank.barrier(dist)
    slowest = multirank.max_over_ranks(mine, dist)
    units = 2 * sum(N + 1 for N, _, _, _ in items)
    units_all = multirank.sum_over_ranks(units, dist)
    print(json.dumps({{
        "rank": rank, "world": world, "max": mx, "sum": sm, "mine": mine, "slowest": slowest,
        "units": units, "units_all": units_all, "rate": multirank.job_rate(units_all, slowest),
        "Ns": [it[0] for it in items], "ab": [[it[1], it[2]] for it in items],
        "csum": [float(np.sum(it[3])) for it in items],
        "batch_Ns": [it[0] for it in batch], "batch_dirs": [it[3] for it in batch],
    }}))
    dist.destroy_process_group()
""")


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    r0, r1 = sorted(outs, key=lambda d: d["rank"])
    for d in (r0, r1):
        assert d["world"] == 2
        assert d["max"] == 2.5 and d["sum"] == 3.0
        assert d["slowest"] == max(r0["mine"], r1["mine"]) and d["slowest"] >= 0.1
        assert d["units_all"] == r0["units"] + r1["units"]
        assert d["rate"] == pytest.approx(d["units_all"] / d["slowest"])
    # rank 0 runs the one-GPU workload; rank 1 a shard of the same shape with its own draws
    import bench
    from paper_1602_02618_gb300 import inputs
    one = bench.workload()
    assert r0["Ns"] == [it[0] for it in one] == r1["Ns"]
    assert r0["ab"] == [[it[1], it[2]] for it in one]
    assert r0["csum"] == [float(np.sum(it[3])) for it in one]
    assert r1["ab"] != r0["ab"] and r1["csum"] != r0["csum"]
    b0 = inputs.batch_workload(8)
    assert r0["batch_Ns"] == [it[0] for it in b0] and r0["batch_dirs"] == [it[3] for it in b0]
    assert r1["batch_Ns"] != r0["batch_Ns"]


def test_reference_arm_under_torchrun():
    """bench.py --impl reference with two ranks: rank 0 times the oracle and prints the only
    line; rank 1 exits 0 without work."""
    pytest.importorskip("torch")
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    # torchrun sets OMP_NUM_THREADS=1; the oracle still runs on, and reports, every core
    assert d["cpu_baseline"]["cores"] == os.cpu_count()
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
