"""Multi-rank timing aggregation of bench.py on CPU (gloo, world size 2).

Each rank matches its own update set; the job's time is the slowest rank's
and its pairs are the sum over ranks.  No GPU is used.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, k = bench.job_totals(1.0 + rank, 100 * (rank + 1), world, device="cpu")
    out[rank] = (t, k)
    tdist.barrier()
    tdist.destroy_process_group()


def test_job_totals_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (2.0, 300.0)


def test_job_totals_single_rank():
    import bench
    assert bench.job_totals(1.5, 42, 1) == (1.5, 42.0)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle on a bounded sample of
    the benchmark workload (here a 1% scale of it) and prints one JSON line
    with the same metric as the GPU arm; no GPU is used."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--scale", "0.01", "--cpu-seconds", "1"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pairs/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_cpu_baseline_small_and_config2_legs():
    """The oracle legs the bench adds to `cpu_baseline`: the N = 1e4 d = 1
    workload as a mean over runs (brute force and ITM agree on K), and the
    N = 1e6 d = 1 / d = 2 workloads on all cores and on one, each with a
    whole-match time extrapolated from a bounded sample."""
    import bench
    sc = bench.cpu_small_configs(reps=2)
    assert sc["runs"] == 2 and sc["K"] > 0 and sc["cores"] >= 1
    assert sc["bf_1core_s"] > 0 and sc["itm_1core_s"] > 0 and sc["itm_all_cores_s"] > 0
    rows = bench.cpu_config2(budget_s=0.2)
    names = [r["workload"] for r in rows]
    assert names == [f"uniform_d{d}_N1e6_a{a}" for d in (1, 2) for a in ("0.01", "1", "100")]
    for r in rows:
        assert r["match_s_all_cores"] > 0 and r["match_s_one_core"] > 0 and r["cores"] >= 1
        assert r["pairs_per_s_all_cores"] >= 0 and "one thread" in r["sample"]
