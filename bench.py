#!/usr/bin/env python3
"""Throughput benchmark of GPU interval tree matching (one JSON line).

A step is one whole match of the workload: sort and tree build over the
subscriptions (ddm_build), the counting pass and scan over all updates
(ddm_plan), then the write pass over ranges of the plan order whose pairs fit
the device pair buffer (ddm_chunk_end_ordered + ddm_write_ordered), every pair
written to HBM.  Inputs
(240 MB for the default workload) are larger than L2, so no flush is needed.

Default workload: d = 3, 5e6 updates + 5e6 subscriptions, centres from 64
Gaussian clusters, log-normal extents, overlap degree 100 (the N = 1e7,
alpha = 100 stress case); about 4.4e10 pairs (354 GB), so the write pass
runs in chunks.

Reported: matched pairs/s (value) and update queries/s; p50/p99 step
latency; the write-pass kernel against the measured HBM roofline; the same
metric end to end with host buffers (inputs copied in, every pair copied
out); the CPU oracle on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle (interval tree matching with
OpenMP over queries on the host cores) on a bounded sample instead.
Multi-GPU (torchrun): one problem split across ranks -- every rank builds the
tree over the whole subscription set and matches a contiguous range of the
update ids, writing global ids (no collective on the data path; the job's
pairs are the sum over ranks, its time the slowest rank's).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_CONFIG = "clustered_d3_N1e7_a100"
# DRAM bytes (read + write) per pair of the write-pass kernel (k_replay), from
# the ncu capture summarised in profiles/k_replay_clustered_d3_scale0.15.md
# (a smaller case of the same workload; traffic scales with pairs written),
# and per id of the compressed output's kernel
# (profiles/k_replay_ids_clustered_d3_scale0.15.md).
TRAFFIC_PER_PAIR = 8.76
TRAFFIC_PER_ID = 5.37
METRIC = "matched pairs/s (N=1e7, alpha=100, d=3)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink n and m (profiling a small case of the same workload)")
    ap.add_argument("--chunk-gb", type=float, default=32.0, help="device pair buffer (GB)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--stage-gb", type=float, default=2.0, help="pinned host staging (GB)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-instances comparison (4,096 problems)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched-instances comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving run")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--no-sweep", action="store_true", help="skip the alpha x N sweep")
    ap.add_argument("--no-compressed", action="store_true",
                    help="skip the compressed-output (subscription ids by column) runs")
    ap.add_argument("--phase", default="all", choices=["all", "build"],
                    help="build: time ddm_build alone (sort + tree) on the workload's "
                         "subscriptions, for profiling the build kernels")
    return ap.parse_args()


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_totals(t_local, pairs_local, world, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time and the pairs of
    all ranks (the only use of the process group; no data-path collective)."""
    if world <= 1:
        return t_local, float(pairs_local)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    k = torch.tensor([float(pairs_local)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(k, op=tdist.ReduceOp.SUM)
    return float(t[0]), float(k[0])


def workload(name, rank=0, world=1, scale=1.0):
    """The named workload; with world > 1 the rank's shard of it: the whole
    subscription set and a contiguous range of the update ids (one problem
    split across ranks, Section IV "Parallelizing ITM").  Returns the arrays
    and the shard's first update id."""
    import numpy as np

    from paper_1309_3458_gb300 import sharded
    from paper_1309_3458_gb300 import workloads as W
    arrays = W.make(name, scale)
    if world == 1:
        return arrays, 0
    b, e = sharded.shard_bounds(arrays[0].shape[1], world)[rank]
    return (np.ascontiguousarray(arrays[0][:, b:e]), np.ascontiguousarray(arrays[1][:, b:e]),
            arrays[2], arrays[3]), b


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples (the JSON line carries their summary); DDM_CLOCKS_DIR keeps them
        out = os.environ.get("DDM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"ddm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                mhz.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def cpu_oracle_sample(arrays, budget_s, one_core: bool = False):
    """Oracle ITM (all host cores) on a bounded sample of the workload: one
    interval tree build over all subscriptions plus a random sample of the
    updates; pairs/s extrapolated to the whole update set (one build, all
    queries at the sampled rate)."""
    import numpy as np

    import oracle
    ulo, uhi, slo, shi = arrays
    m = ulo.shape[1]
    threads = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(123)
    sub = lambda idx: (np.ascontiguousarray(ulo[:, idx]), np.ascontiguousarray(uhi[:, idx]))
    # probe: build + 256 queries, to size the sample
    probe = np.sort(rng.choice(m, min(m, 256), replace=False))
    tm = []
    oracle.itm_count(*sub(probe), slo, shi, threads=threads, timings=tm)
    t_build, per_q = tm[0], max(1e-7, tm[1] / len(probe))
    q = int(min(m, max(256, (budget_s - t_build) / per_q)))
    sample = np.sort(rng.choice(m, q, replace=False))
    tm = []
    t0 = time.perf_counter()
    K, _, _ = oracle.itm_count(*sub(sample), slo, shi, threads=threads, timings=tm)
    wall = time.perf_counter() - t0
    t_build, t_q = tm
    t_all = t_build + t_q * m / q
    out = {"value": K * m / q / t_all, "unit": "pairs/s", "cores": threads, "kind": "oracle",
           "sample": (f"interval tree (AVL) build over all {slo.shape[1]} subscriptions "
                      f"({t_build:.2f} s) + {q} of {m} updates queried with OpenMP on "
                      f"{threads} threads ({t_q:.2f} s, {K} pairs); rate extrapolated to all "
                      f"updates"),
           "queries_per_s": m / t_all, "seconds": wall}
    if one_core:
        # the sequential ITM (one thread), on a quarter of the sample
        s1 = np.sort(rng.choice(m, max(64, q // 4), replace=False))
        tm = []
        K1, _, _ = oracle.itm_count(*sub(s1), slo, shi, threads=1, timings=tm)
        t1 = tm[0] + tm[1] * m / len(s1)
        out["one_core"] = {"value": K1 * m / len(s1) / t1, "unit": "pairs/s",
                           "sample": f"{len(s1)} of {m} updates on one thread, same extrapolation",
                           "queries_per_s": m / t1}
    return out


def cpu_small_configs(reps: int = 30):
    """The oracle on the N = 1e4, d = 1 workload: brute force (Alg. 2) on one
    thread and the interval tree (Algs. 4-5, build included) on one thread
    and on all host cores, each the mean of `reps` runs (the paper reports
    the mean of 30)."""
    import numpy as np

    import oracle
    from paper_1309_3458_gb300 import workloads as W
    a = W.make("uniform_d1_N1e4_a1")
    threads = len(os.sched_getaffinity(0))
    out = {"workload": "uniform_d1_N1e4_a1", "runs": reps}
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        K = oracle.bf(*a, pairs=False)[0]
        ts.append(time.perf_counter() - t0)
    out["bf_1core_s"] = float(np.mean(ts))
    for name, th in (("itm_1core_s", 1), ("itm_all_cores_s", threads)):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            Ki, _, _ = oracle.itm_count(*a, threads=th)
            ts.append(time.perf_counter() - t0)
            assert Ki == K
        out[name] = float(np.mean(ts))
    out["K"] = int(K)
    out["cores"] = threads
    return out


def cpu_config2(budget_s: float = 2.0):
    """The oracle's interval tree (Algs. 4-5) on the N = 1e6 workloads (d = 1
    and 2, alpha = 0.01, 1, 100) on all host cores and on one: one build
    over all subscriptions plus a sample of the updates sized to about
    `budget_s`, the rate extrapolated to all updates (cpu_oracle_sample);
    match_s is the extrapolated time of the whole matching, build included.
    Brute force is not timed here: 2.5e11 segment tests per workload."""
    from paper_1309_3458_gb300 import workloads as W
    out = []
    for d in (1, 2):
        for tag in ("0.01", "1", "100"):
            name = f"uniform_d{d}_N1e6_a{tag}"
            a = W.make(name)
            m = a[0].shape[1]
            r = cpu_oracle_sample(a, budget_s, one_core=True)
            out.append({"workload": name, "cores": r["cores"],
                        "match_s_all_cores": m / r["queries_per_s"],
                        "match_s_one_core": m / r["one_core"]["queries_per_s"],
                        "pairs_per_s_all_cores": r["value"],
                        "pairs_per_s_one_core": r["one_core"]["value"],
                        "sample": r["sample"] + "; " + r["one_core"]["sample"]})
    return out


def batched_section(reps: int = 3):
    """Batched instances: 4,096 independent d = 2 problems with log-uniform
    sizes in [100, 1e5] extents (alpha = 1 each).  Plain: one ddm_match per
    instance (each with its own host synchronisation).  Batched: the
    autotuned ddm_batch_match_async recorded once into a CUDA graph and
    replayed.  Both produce the same pairs (checked by count)."""
    import numpy as np
    import torch

    import paper_1309_3458_gb300 as ddm
    from paper_1309_3458_gb300 import autotune as AT
    from paper_1309_3458_gb300 import workloads as W
    inst = W.batched_instances(4096, d=2, alpha=1.0, size_lo=100, size_hi=100_000, seed=0)
    ulo, uhi, uoff, slo, shi, soff = W.concat_instances(inst)
    ctx = ddm.ddm_create(torch.cuda.current_device())
    try:
        # plain per-instance calls
        per = [tuple(torch.from_numpy(a).cuda() for a in x) for x in inst]
        Ks = [ddm.ddm_count(ctx, *u) for u in per]
        K = int(sum(Ks))
        buf = torch.empty((K + 1, 2), dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()

        def plain():
            o = 0
            for u, k in zip(per, Ks):
                ddm.ddm_match(ctx, *u, buf[o:])
                o += k

        plain()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            plain()
        ev[1].record(stream)
        torch.cuda.synchronize()
        plain_ms = ev[0].elapsed_time(ev[1]) / reps

        # batched
        U = tuple(torch.from_numpy(a).cuda() for a in (ulo, uhi, slo, shi))
        uo = torch.from_numpy(uoff.astype(np.int64)).cuda()
        so = torch.from_numpy(soff.astype(np.int64)).cuda()
        pof = torch.empty(len(inst) + 1, dtype=torch.int64, device="cuda")
        kd = torch.zeros(1, dtype=torch.int64, device="cuda")
        ed = torch.zeros(1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(stream)

        def batched():
            ddm.ddm_batch_match_async(ctx, U[0], U[1], uo, U[2], U[3], so, buf, pof, kd, ed,
                                      stream=s)

        with torch.cuda.stream(s):
            best, table = AT.autotune(ctx, batched, stream=s)
            batched()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            batched()
        kd.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):   # replay() launches on the current stream
            g.replay()
        torch.cuda.synchronize()
        Kb, err = int(kd[0]), int(ed[0])
        ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(s):
            ev2[0].record(s)
            for _ in range(reps * 4):
                g.replay()
            ev2[1].record(s)
        torch.cuda.synchronize()
        batched_ms = ev2[0].elapsed_time(ev2[1]) / (reps * 4)
        return {"workload": "4096 instances, d=2, alpha=1, sizes log-uniform [100, 1e5]",
                "extents": int(uoff[-1] + soff[-1]), "K": K, "K_batched": Kb, "err": err,
                "plain_ms": plain_ms, "batched_ms": batched_ms,
                "plain_pairs_per_s": K / plain_ms * 1e3,
                "batched_pairs_per_s": Kb / batched_ms * 1e3,
                "speedup": plain_ms / batched_ms, "tuning": best,
                "tuning_table_ms": [[round(t, 3), c] for t, c in table]}
    finally:
        ddm.ddm_destroy(ctx)


def serving_section(seconds: float = 2.0, slots: int = 4, saturated_seconds: float = 1.0):
    """Serving: d = 2, 1e6 resident subscription regions (side 1e3, i.e.
    alpha = 1 at N = 1e6) moving every 10 ms by a Gaussian random walk
    (sigma = 1e-3 L, reflected); 64 federates send match requests with
    Poisson arrivals (2,000 per second in total) and update-set sizes
    log-uniform in [1e3, 1e6]; continuous batching over `slots` streams with
    admission by a device-memory budget.  The federates' update sets are on
    the device when their requests arrive.

    Three runs: the real-time schedule (latency percentiles), a saturated
    schedule whose requests all wait at t = 0 (throughput), and the same
    saturated requests served plainly -- one ddm_plan + ddm_write per
    request, one after another."""
    import torch

    import paper_1309_3458_gb300 as ddm
    from paper_1309_3458_gb300 import serving as S
    d, n, l = 2, 1_000_000, 1000.0
    g = torch.Generator(device="cuda")
    g.manual_seed(2026)
    lo = (torch.rand((d, n), generator=g, device="cuda") * (S.L - l)).contiguous()
    hi = (lo + l).contiguous()
    # regions move by about their own side per step: rebuilding (re-sorting)
    # the idle version every step beats refitting an ageing order
    regions = S.ResidentRegions(lo, hi, rebuild_every=1)
    state = {"lo": lo, "hi": hi}
    mg = torch.Generator(device="cuda")
    mg.manual_seed(7)

    def mover(step):
        state["lo"], state["hi"] = S.random_walk(state["lo"], state["hi"], 1000.0, mg)
        return state["lo"], state["hi"]

    def materialise(reqs):
        sets = [S.request_updates(r.seed, r.size, d, l) for r in reqs]
        torch.cuda.synchronize()
        return sets

    def attach(reqs, sets):
        for r, (a, b) in zip(reqs, sets):
            r.lo, r.hi = a, b

    sched = S.poisson_schedule(rate=2000.0, duration=seconds, federates=64, size_lo=1000,
                               size_hi=1_000_000, seed=1)
    sat = S.poisson_schedule(rate=2000.0, duration=saturated_seconds, federates=64,
                             size_lo=1000, size_hi=1_000_000, seed=2)
    for r in sat:
        r.arrival = 0.0
    warm = S.poisson_schedule(rate=2000.0, duration=0.25, federates=64, size_lo=1000,
                              size_hi=1_000_000, seed=3)
    sched_sets, sat_sets, warm_sets = materialise(sched), materialise(sat), materialise(warm)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.4)
    srv = S.Server(regions, l, slots=slots, budget_bytes=budget, pair_capacity=1 << 26)
    try:
        srv.warm_up()
        attach(warm, warm_sets)     # untimed: first use of every step of the loop
        srv.run(warm, mover=mover, step_s=0.010)
        attach(sched, sched_sets)
        t0 = time.perf_counter()
        done = srv.run(sched, mover=mover, step_s=0.010)
        wall = time.perf_counter() - t0
        rt_launches = srv.launches
        attach(sat, sat_sets)
        srv.launches = 0
        t0 = time.perf_counter()
        sdone = srv.run(sat, mover=None)     # fixed version: plain must find the same pairs
        sat_wall = time.perf_counter() - t0
        sat_launches = srv.launches
    finally:
        srv.close()
    # plain: one ddm_plan + ddm_write per request, one after another
    ctx = ddm.ddm_create(torch.cuda.current_device())
    buf = torch.empty((1 << 26, 2), dtype=torch.int32, device="cuda")
    try:
        ddm.ddm_attach(ctx, regions.ctx[regions.active])
        for a, b in sat_sets[:3]:     # warm-up: size the context's workspace
            ddm.ddm_plan(ctx, a, b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain_K = 0
        for r, (a, b) in zip(sat, sat_sets):
            k = ddm.ddm_plan(ctx, a, b)
            ddm.ddm_write(ctx, 0, r.size, buf)
            plain_K += k
        torch.cuda.synchronize()
        plain_wall = time.perf_counter() - t0
    finally:
        ddm.ddm_destroy(ctx)
        regions.close()
    out = S.summary(done, wall)
    out["launches"] = rt_launches
    sq = sum(r.size for r in sdone)
    sK = sum(r.K for r in sdone)
    out["saturated"] = {"requests": len(sdone), "wall_s": sat_wall, "launches": sat_launches,
                        "queries_per_s": sq / sat_wall, "pairs_per_s": sK / sat_wall,
                        "p50_ms": S.summary(sdone, sat_wall)["p50_ms"]}
    out["plain_one_at_a_time"] = {"requests": len(sat), "wall_s": plain_wall,
                                  "queries_per_s": sq / plain_wall,
                                  "pairs_per_s": plain_K / plain_wall,
                                  "same_pairs": plain_K == sK}
    out["served_over_plain"] = plain_wall / sat_wall
    out.update({"workload": "d=2, 1e6 moving regions, 64 federates, 2000 req/s Poisson, "
                            "sizes log-uniform [1e3, 1e6]",
                "policy": "rebuild the idle version every step",
                "rebuilds": regions.rebuilds, "refits": regions.refits,
                "slots": slots, "budget_gb": budget / 1e9, "offered_s": seconds,
                "steps": max(r.step for r in done) if done else 0})

    # The same real-time schedule under the configured in-place refit per
    # step: refit only, and refit with a rebuild when a probe finds the
    # refitted tree slower than `adaptive` times its post-rebuild speed.
    out["other_policies"] = {}
    for pname, kw in (("refit_every_step", dict(rebuild_every=0)),
                      ("refit_every_step_rebuild_when_1.5x_slower",
                       dict(rebuild_every=0, adaptive=1.5))):
        g.manual_seed(2026)
        lo = (torch.rand((d, n), generator=g, device="cuda") * (S.L - l)).contiguous()
        hi = (lo + l).contiguous()
        state.update(lo=lo, hi=hi)
        mg.manual_seed(7)
        reg = S.ResidentRegions(lo, hi, **kw)
        sched2 = S.poisson_schedule(rate=2000.0, duration=seconds, federates=64, size_lo=1000,
                                    size_hi=1_000_000, seed=1)
        warm2 = S.poisson_schedule(rate=2000.0, duration=0.25, federates=64, size_lo=1000,
                                   size_hi=1_000_000, seed=3)
        srv2 = S.Server(reg, l, slots=slots, budget_bytes=budget, pair_capacity=1 << 26)
        try:
            srv2.warm_up()
            attach(warm2, warm_sets)
            srv2.run(warm2, mover=mover, step_s=0.010)
            attach(sched2, sched_sets)
            t0 = time.perf_counter()
            done2 = srv2.run(sched2, mover=mover, step_s=0.010)
            wall2 = time.perf_counter() - t0
        finally:
            srv2.close()
            reg.close()
        o2 = S.summary(done2, wall2)
        o2.update({"rebuilds": reg.rebuilds, "refits": reg.refits,
                   "steps": max(r.step for r in done2) if done2 else 0})
        if reg.tests_ratio:
            o2["probe_tests_ratio_max"] = max(reg.tests_ratio)
        out["other_policies"][pname] = o2
    return out


# ALU pipe of one SM: 64 lanes (16 per sub-partition; ncu's own ALU-pipe
# peak, 0.5 warp instructions per cycle per sub-partition); a float compare is
# one lane operation.  The peak multiplies this by the device's SM count and
# the median SM clock sampled during the timed region (the 2,070 MHz maximum
# when no sample exists).
ALU_LANES_PER_SM = 64
MAX_SM_MHZ = 2070.0


def alu_peak_gcmp(sms, sm_mhz):
    return sms * ALU_LANES_PER_SM * (sm_mhz or MAX_SM_MHZ) / 1e3


def count_roofline(leaf_tests, d, count_ms, steps, sms, sm_mhz):
    """The count pass (`k_packets`, issue / ALU bound): segment comparisons
    the tree walk makes -- 2d per tested subscription, 32 subscriptions per
    (query, leaf) test, counted by the kernel itself -- per second of
    ddm_plan (update sort + count pass + scans; the count pass is about 97%
    of it), against the ALU pipe's compare rate."""
    sec = sum(a.elapsed_time(b) for a, b in count_ms) / 1e3 / max(1, steps)
    cmp = float(leaf_tests) * 32 * 2 * d
    achieved = cmp / sec / 1e9 if sec > 0 else 0.0
    peak = alu_peak_gcmp(sms, sm_mhz)
    return {"bound": "alu", "kernel": "k_packets (count pass, ddm_plan)", "achieved": achieved,
            "peak": peak, "unit": "Gcmp/s", "frac": achieved / peak,
            "leaf_tests": int(leaf_tests), "plan_ms_per_step": 1e3 * sec,
            "peak_source": f"{sms} SMs x {ALU_LANES_PER_SM} ALU lanes x "
                           f"{sm_mhz or MAX_SM_MHZ:.0f} MHz ("
                           + ("median sampled SM clock)" if sm_mhz else "maximum SM clock)")}


def query_bytes(d, n, m, K):
    """Algorithmic bytes of one whole match: every input extent read once
    (8 d bytes: lower and upper bound per dimension), every pair written once
    (8 bytes), and the tree build (three passes of 12 bytes per subscription:
    key, id and bound)."""
    return {"inputs": 8 * d * (n + m), "pairs": 8 * K, "build": 36 * n}


def configs_section(skip: str, reps: int = 3):
    """Every other named workload (the paper's Section V shapes: d = 1 at
    N = 1e4, d = 1 and 2 at N = 1e6 for alpha = 0.01, 1, 100): one full
    ddm_match each (build, count, write, pairs in a device buffer), median of
    `reps` timed with CUDA events after one warm-up."""
    import torch

    import paper_1309_3458_gb300 as ddm
    from paper_1309_3458_gb300 import workloads as W
    ctx = ddm.ddm_create(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = []
    try:
        for name in W.CONFIGS:
            if name == skip:
                continue
            U = [torch.from_numpy(x).cuda() for x in W.make(name)]
            K = ddm.ddm_count(ctx, *U)
            buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
            ddm.ddm_match(ctx, *U, buf)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ddm.ddm_match(ctx, *U, buf)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ts.sort()
            ms = ts[len(ts) // 2]
            out.append({"workload": name, "K": K, "ms": round(ms, 4),
                        "pairs_per_s": K / (ms / 1e3) if ms > 0 else None,
                        "queries_per_s": U[0].shape[1] / (ms / 1e3) if ms > 0 else None})
            del buf, U
    finally:
        ddm.ddm_destroy(ctx)
    return out


def sweep_section(reps: int = 3):
    """The shape of the paper's Fig. 7 (Section V): d = 1 uniform workloads,
    N = n + m from the paper's 5e4 and 5e5 up to 5e7, overlapping degree
    alpha in {1, 10, 100}; one full match (build, count, write) per point,
    median of `reps` timed with CUDA events after one warm-up.  At the
    paper's sizes a call is bound by its launches and its host
    synchronisation; from N = 5e6 on the time follows K."""
    import torch

    import paper_1309_3458_gb300 as ddm
    from paper_1309_3458_gb300 import workloads as W
    ctx = ddm.ddm_create(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = []
    try:
        for N in (50_000, 500_000, 5_000_000, 50_000_000):
            for alpha in (1.0, 10.0, 100.0):
                a = W.uniform_fixed_length(N - N // 2, N // 2, 1, alpha, seed=7)
                U = [torch.from_numpy(x).cuda() for x in a]
                K = ddm.ddm_count(ctx, *U)
                buf = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda")
                ddm.ddm_match(ctx, *U, buf)
                ts = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ddm.ddm_match(ctx, *U, buf)
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ts.sort()
                ms = ts[len(ts) // 2]
                out.append({"N": N, "alpha": alpha, "K": K, "ms": round(ms, 4),
                            "pairs_per_s": K / ms * 1e3, "queries_per_s": (N // 2) / ms * 1e3})
                del buf, U
    finally:
        ddm.ddm_destroy(ctx)
    return out


def build_phase(args, ddm):
    """ddm_build alone (validation, class keys, radix sort, re-sorts, tree
    build) on the workload's subscription set."""
    import torch
    from paper_1309_3458_gb300 import workloads as W
    a = W.make(args.config, args.scale)
    lo, hi = torch.from_numpy(a[2]).cuda(), torch.from_numpy(a[3]).cuda()
    ctx = ddm.ddm_create(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    try:
        for _ in range(args.warmup):
            ddm.ddm_build(ctx, lo, hi)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ddm.ddm_debug_launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            ddm.ddm_build(ctx, lo, hi)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(1, args.steps)
        launches = (ddm.ddm_debug_launch_count() - l0) // max(1, args.steps)
    finally:
        ddm.ddm_destroy(ctx)
    n = lo.shape[1]
    return {"phase": "build", "workload": args.config if args.scale == 1.0 else
            f"{args.config}@{args.scale}", "n_sub": n, "d": lo.shape[0], "ms_per_build": ms,
            "subscriptions_per_s": n / (ms / 1e3), "gpu_launches": int(launches)}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    arrays, _ = workload(args.config, scale=args.scale)
    res = []
    for _ in range(args.warmup + args.steps):
        res.append(cpu_oracle_sample(arrays, args.cpu_seconds / max(1, args.steps)))
    timed = res[args.warmup:]
    v = statistics.mean(r["value"] for r in timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(r["seconds"] for r in timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": args.config},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": timed[0]["cores"],
                             "kind": "oracle", "sample": timed[0]["sample"]},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as tdist

    import paper_1309_3458_gb300 as ddm
    torch.cuda.set_device(local)
    if args.batched_only:
        print(json.dumps({"batched": batched_section()}), flush=True)
        return
    if args.serving_only:
        print(json.dumps({"serving": serving_section(args.serving_seconds)}), flush=True)
        return
    if args.phase == "build":
        print(json.dumps(build_phase(args, ddm)), flush=True)
        return
    if world > 1:
        tdist.init_process_group("nccl")

    def barrier():
        if world > 1:
            tdist.barrier()

    arrays, upd_base = workload(args.config, rank, world, args.scale)
    d, m = arrays[0].shape
    n = arrays[2].shape[1]
    dev = tuple(torch.from_numpy(a).cuda() for a in arrays)
    ctx = ddm.ddm_create(local)
    ddm.ddm_set_update_id_base(ctx, upd_base)   # this rank's pairs carry global update ids
    cap = int(args.chunk_gb * 1e9) // 8
    pairs = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    write_ms, write_bytes, write_pairs, plan_ms, count_ms = [], [], [], [], []
    chunks = [0]
    tests = [0]

    def step(record=False):
        if record:
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
        ddm.ddm_build(ctx, dev[2], dev[3])
        if record:
            ab = torch.cuda.Event(enable_timing=True)
            ab.record(stream)
        K = ddm.ddm_plan(ctx, dev[0], dev[1])
        if record:
            a1.record(stream)
            plan_ms.append((a0, a1))
            count_ms.append((ab, a1))
            tests[0] = ddm.ddm_plan_stats(ctx)
        b = 0
        chunks[0] = 0
        while b < m:
            e = ddm.ddm_chunk_end_ordered(ctx, b, cap)
            chunks[0] += 1
            if record:
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
            k = ddm.ddm_write_ordered(ctx, b, e, pairs)
            if record:
                s1.record(stream)
                write_ms.append((s0, s1))
                write_bytes.append(8 * k)
                write_pairs.append(k)
            b = e
        return K

    K = 0
    for _ in range(args.warmup):
        K = step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    l0 = ddm.ddm_debug_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with Clocks(local) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            K = step(record=True)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = (ddm.ddm_debug_launch_count() - l0) // args.steps
    total_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    t_local = total_ms / 1e3
    pairs_local = K * args.steps
    t_job, pairs_job = job_totals(t_local, pairs_local, world, device="cuda")
    _, queries_job = job_totals(t_local, m * args.steps, world, device="cuda")
    wtimes = [a.elapsed_time(b) for a, b in write_ms]
    write_s = sum(wtimes) / 1e3
    write_gbs = sum(write_bytes) / write_s / 1e9 if write_s > 0 else 0.0

    peaks = {}
    if os.path.exists(PEAKS):
        peaks = json.load(open(PEAKS))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    # ---- compressed output (Section III: M stored by columns) ----
    # The same step, writing only each pair's subscription id (4 bytes) into
    # the same device buffer, plus the plan order (the update of each column)
    # and the column offsets.
    ids_all = pairs.view(-1)
    cap_ids = ids_all.shape[0]
    order_d = torch.empty(m, dtype=torch.int32, device="cuda")
    ooff_d = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    compressed = None
    if not args.no_compressed:
        cw_ms, cw_bytes, cw_ids = [], [], []

        def step_ids(c, record=False, cap_c=cap_ids, buf=ids_all):
            ddm.ddm_build(c, dev[2], dev[3])
            Kc = ddm.ddm_plan(c, dev[0], dev[1])
            ddm.ddm_plan_order(c, order_d, ooff_d)
            b = 0
            while b < m:
                e = ddm.ddm_chunk_end_ordered(c, b, cap_c)
                if record:
                    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    s0.record(stream)
                k = ddm.ddm_write_ordered_ids(c, b, e, buf)
                if record:
                    s1.record(stream)
                    cw_ms.append((s0, s1))
                    cw_bytes.append(4 * k)
                    cw_ids.append(k)
                b = e
            return Kc

        for _ in range(args.warmup):
            step_ids(ctx)
        torch.cuda.synchronize()
        barrier()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            Kc = step_ids(ctx, record=True)
        c1.record(stream)
        torch.cuda.synchronize()
        barrier()
        c_s = c0.elapsed_time(c1) / 1e3
        t_c, k_c = job_totals(c_s, Kc * args.steps, world, device="cuda")
        cws = sum(a.elapsed_time(b) for a, b in cw_ms) / 1e3
        c_gbs = sum(cw_bytes) / cws / 1e9 if cws > 0 else 0.0
        compressed = {
            "value": k_c / t_c,
            "unit": "pairs/s", "ms_per_step": 1e3 * c_s / args.steps,
            "write_ms_per_step": 1e3 * cws / args.steps, "K": Kc,
            "chunks": len(cw_ids) // max(1, args.steps),
            "output": "subscription ids (uint32) in plan order + plan order (uint32) + column "
                      "offsets (uint64): the intersection matrix by columns",
            "roofline": {"bound": "hbm", "kernel": "k_replay (ddm_write_ordered_ids)",
                         "achieved": c_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": c_gbs / hbm_peak, "peak_source": peak_src,
                         "traffic": TRAFFIC_PER_ID * sum(cw_ids) / max(1, len(cw_ids)),
                         "bytes_per_launch": "4*(ids in chunk): each id written once"}}

    # ---- end to end with host buffers ----
    # Inputs are copied from pinned host memory every step and every pair is
    # copied back to pinned host memory.  The device pair buffer is split in
    # two halves: while one half's pairs travel to the host on a copy stream,
    # the next chunk is written into the other half.  Two contexts alternate
    # between steps, so that a step's build and count run while the previous
    # step's last pairs are still being copied out.
    e2e = e2e_compressed = None
    if not args.no_e2e:
        host = [torch.from_numpy(a).pin_memory() for a in arrays]
        stage = torch.empty((int(args.stage_gb * 1e9) // 8, 2), dtype=torch.int32).pin_memory()
        h2d = sum(a.nbytes for a in arrays)
        e2e_steps = args.e2e_steps or max(1, min(args.steps, 3))
        half = cap // 2
        bufs = (pairs[:half], pairs[half:2 * half])
        half_ids = cap_ids // 2
        bufs_ids = (ids_all[:half_ids], ids_all[half_ids:2 * half_ids])
        stage_ids = stage.view(-1)
        order_h = torch.empty(m, dtype=torch.int32).pin_memory()
        ooff_h = torch.empty(m + 1, dtype=torch.int64).pin_memory()
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        ctxs = (ctx, ddm.ddm_create(local))
        chunk_no = [0]

        def e2e_run(nsteps, ids=False):
            Ke = 0
            for st in range(nsteps):
                c = ctxs[st % 2]
                for t_dev, t_host in zip(dev, host):
                    t_dev.copy_(t_host, non_blocking=True)
                ddm.ddm_build(c, dev[2], dev[3])
                Ke = ddm.ddm_plan(c, dev[0], dev[1])
                if ids:   # the columns' updates and offsets, then the ids chunk by chunk
                    stream.wait_event(copied[0])
                    stream.wait_event(copied[1])
                    ddm.ddm_plan_order(c, order_d, ooff_d)
                    planned = torch.cuda.Event()
                    planned.record(stream)
                    copy_stream.wait_event(planned)
                    with torch.cuda.stream(copy_stream):
                        order_h.copy_(order_d, non_blocking=True)
                        ooff_h.copy_(ooff_d, non_blocking=True)
                b = 0
                while b < m:
                    e = ddm.ddm_chunk_end_ordered(c, b, half_ids if ids else half)
                    i = chunk_no[0]
                    buf = (bufs_ids if ids else bufs)[i % 2]
                    stream.wait_event(copied[i % 2])      # that half's previous pairs are out
                    k = (ddm.ddm_write_ordered_ids if ids else ddm.ddm_write_ordered)(c, b, e, buf)
                    written = torch.cuda.Event()
                    written.record(stream)
                    copy_stream.wait_event(written)
                    st_buf = stage_ids if ids else stage
                    with torch.cuda.stream(copy_stream):
                        o = 0
                        while o < k:
                            n_c = min(st_buf.shape[0], k - o)
                            st_buf[:n_c].copy_(buf[o:o + n_c], non_blocking=True)
                            o += n_c
                        copied[i % 2].record(copy_stream)
                    b, chunk_no[0] = e, i + 1
            stream.wait_stream(copy_stream)
            torch.cuda.synchronize()
            return Ke

        for _ in range(2):   # size the second context's workspace and record arena
            ddm.ddm_build(ctxs[1], dev[2], dev[3])
            ddm.ddm_plan(ctxs[1], dev[0], dev[1])
        e2e_run(1)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Ke = e2e_run(e2e_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = e0.elapsed_time(e1) / 1e3
        e2e = {"value": Ke * e2e_steps / te * (world if world > 1 else 1), "unit": "pairs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * Ke),
               "steps": e2e_steps}
        if not args.no_compressed:
            e2e_run(1, ids=True)
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            Ke = e2e_run(e2e_steps, ids=True)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            te = e0.elapsed_time(e1) / 1e3
            e2e_compressed = {
                "value": Ke * e2e_steps / te * (world if world > 1 else 1), "unit": "pairs/s",
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(4 * Ke + order_h.nbytes + ooff_h.nbytes),
                "steps": e2e_steps, "output": "compressed (ids by column)"}
        ddm.ddm_destroy(ctxs[1])
        del host, stage

    ddm.ddm_destroy(ctx)
    if rank != 0:
        return

    batched = None
    if not args.no_batched and world == 1:
        del pairs
        torch.cuda.empty_cache()
        batched = batched_section()

    serving = None
    if not args.no_serving and world == 1:
        torch.cuda.empty_cache()
        serving = serving_section(args.serving_seconds)

    sweep = others = None
    if not args.no_sweep and world == 1:
        sweep = sweep_section()
        others = configs_section(args.config)

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_oracle_sample(arrays, args.cpu_seconds, one_core=True)
        cpu.pop("seconds", None)
        cpu["small_configs"] = cpu_small_configs()
        cpu["config2"] = cpu_config2()

    clocks = clk.summary()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    qb = query_bytes(d, n, m, K)
    qbytes = qb["inputs"] + qb["pairs"]
    sbytes = qbytes + qb["build"]
    q_s = (sum(a.elapsed_time(b) for a, b in count_ms) / 1e3 + write_s) / args.steps
    step_s = total_ms / 1e3 / args.steps
    line = {
        "metric": METRIC,
        "value": pairs_job / t_job,
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.config if args.scale == 1.0 else f"{args.config}@{args.scale}",
                   "d": d, "n_sub": n, "m_upd": m, "K": K,
                   "parallelism": "one problem, update ids split into %d contiguous range%s "
                                  "(rank 0's: %d updates, K = %d)" % (world, "s" if world > 1 else "",
                                                                     m, K),
                   "chunk_pairs": cap, "chunks": chunks[0], "l2": "inputs %.0f MB (%s L2, no flush)" % (
                       sum(a.nbytes for a in arrays) / 1e6,
                       "larger than" if sum(a.nbytes for a in arrays) > 129e6 else "within")},
        "queries_per_s": queries_job / t_job,
        "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "roofline": {"bound": "hbm", "kernel": "k_replay (ddm_write_ordered)",
                     "achieved": write_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": write_gbs / hbm_peak,
                     "traffic": (TRAFFIC_PER_PAIR * sum(write_pairs) / max(1, len(write_pairs))
                                 if TRAFFIC_PER_PAIR else None),
                     "traffic_note": "DRAM bytes per launch, scaled by pairs written from an ncu "
                                     "capture of the same workload at scale 0.15",
                     "peak_source": peak_src,
                     "bytes_per_launch": "8*(pairs in chunk): each pair written once",
                     "note": "the HBM-bound kernel of the step; the whole query and the whole "
                             "step are in roofline_query and roofline_step, the ALU-bound count "
                             "pass in roofline_count",
                     "write_ms_per_step": 1e3 * write_s / args.steps},
        "roofline_query": {"bound": "hbm", "what": "ddm_plan + ddm_write_ordered (update sort, "
                                                    "count pass, scans, write pass)",
                           "achieved": qbytes / q_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                           "frac": qbytes / q_s / 1e9 / hbm_peak, "peak_source": peak_src,
                           "bytes": qbytes, "ms": 1e3 * q_s,
                           "bytes_formula": "8*d*(n+m) + 8*K"},
        "roofline_step": {"bound": "hbm", "what": "ms_per_step (build + plan + write)",
                          "achieved": sbytes / step_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                          "frac": sbytes / step_s / 1e9 / hbm_peak, "peak_source": peak_src,
                          "bytes": sbytes, "bytes_formula": "8*d*(n+m) + 8*K + 36*n"},
        "roofline_count": count_roofline(tests[0], d, count_ms, args.steps, n_sms,
                                         clocks["sm_mhz"] if clocks else None),
        "phases_ms_per_step": {
            "build_and_count": sum(a.elapsed_time(b) for a, b in plan_ms) / args.steps,
            "write": 1e3 * write_s / args.steps,
            "count_bound": "alu (issue-bound tree walk, see profiles/)"},
        "e2e": e2e,
        "compressed": compressed,
        "e2e_compressed": e2e_compressed,
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "clocks": clocks,
        "batched": batched,
        "serving": serving,
        "alpha_n_sweep": sweep,
        "other_configs": others,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
