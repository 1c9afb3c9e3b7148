"""Serving loop: continuous batching of match requests against resident,
moving subscription regions.

The paper's dynamic setting (Section IV, "Dynamic interval management"):
extents move, and each update set queries the subscription tree again.  Here
the subscriptions stay resident on the device in two tree versions; every
movement step refits the idle version in place (``ddm_refit``: same order,
new per-node bounds) and makes it the active one.  Match requests (update
sets of any size) arrive over time; whenever a slot (context, stream,
buffers) is free, the waiting requests that fit its limits and the memory
budget are admitted together, matched against the version active at
admission in one plan and one write pass over their concatenated update
sets, and pin that version until they complete.  Slots run concurrently, so
requests admitted while others run overlap on the GPU.  A version is refitted
only when no request pins it, and the queries of one update set are
independent of the others in the launch (Section IV), so a request's result
does not depend on what else runs.

Host orchestration only: every step of the matching runs in libddm's
kernels.  Update sets and movement are synthesised on the device with seeded
torch generators (workload generation, not matching arithmetic).
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass
from typing import Any, Deque, Dict, List, Optional

import numpy as np

import paper_1309_3458_gb300 as ddm

L = 1.0e6


def request_updates(seed: int, size: int, d: int, l: float, device="cuda"):
    """Update set of a request: lower bounds uniform in [0, L - l) (float32),
    upper = fl32(lower + fl32(l)); reproducible from (seed, size)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lo = torch.rand((d, size), generator=g, device=device, dtype=torch.float32) * float(L - l)
    hi = lo + torch.tensor(l, dtype=torch.float32, device=device)
    return lo.contiguous(), hi.contiguous()


def random_walk(lo, hi, sigma: float, gen):
    """One movement step: every region moves by N(0, sigma^2) per axis,
    reflected at the borders of [0, L - length] (length unchanged)."""
    import torch
    length = hi - lo
    top = (L - length)
    x = lo + sigma * torch.randn(lo.shape, generator=gen, device=lo.device, dtype=torch.float32)
    x = torch.where(x < 0, -x, x)
    x = torch.where(x > top, 2 * top - x, x)
    x = torch.clamp(x, min=torch.zeros_like(top), max=top)
    return x.contiguous(), (x + length).contiguous()


class ResidentRegions:
    """Subscriptions kept on the device in two tree versions.

    A movement step brings the idle version up to date and activates it,
    by an in-place refit (same order, new node bounds) or, every
    `rebuild_every`-th step, by a full rebuild (re-sort); with `adaptive`,
    by a refit every step followed by a rebuild when a probe finds the
    refitted tree too slow.  A refit keeps the
    result exact, but the order ages: the regions of a leaf drift apart, its
    bounding box grows and the queries test more candidates, so the order is
    renewed periodically (`rebuild_every` = 0: refit only; 1: rebuild every
    step)."""

    def __init__(self, lo, hi, keep_history: bool = False, rebuild_every: int = 1,
                 adaptive: float = 0.0, probe_size: int = 4096, probe_seed: int = 99):
        """adaptive > 0 (with rebuild_every = 0): refit every step in place, then
        measure the refitted tree with a fixed probe update set (its (query,
        leaf) tests per query, ddm_plan_stats); when that exceeds `adaptive`
        times the value measured after the last rebuild, rebuild the version
        instead (the order has aged too far)."""
        import torch
        self.d, self.n = lo.shape
        self.ctx = [ddm.ddm_create(lo.device.index or 0) for _ in range(2)]
        self.adaptive = adaptive
        self.probe_ctx = None
        self.tests_ratio: List[float] = []
        if adaptive > 0:
            side = float((hi[:, :1] - lo[:, :1]).max().item())
            self.probe = request_updates(probe_seed, probe_size, self.d, side, device=lo.device)
            self.probe_ctx = ddm.ddm_create(lo.device.index or 0)
            self.base_tests = [0.0, 0.0]
        self.pos = [(lo.clone(), hi.clone()), (lo.clone(), hi.clone())]
        self.stream = torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            for v in range(2):
                ddm.ddm_build(self.ctx[v], self.pos[v][0], self.pos[v][1], stream=self.stream)
        self.step_of = [0, 0]
        self.active = 0
        self.refs = [0, 0]
        self.cv = threading.Condition()
        self.history = {0: (lo.clone(), hi.clone())} if keep_history else None
        self.rebuild_every = rebuild_every
        self.rebuilds = self.refits = 0
        if self.probe_ctx is not None:
            for v in range(2):
                self.base_tests[v] = self._probe(v)

    def _probe(self, v) -> float:
        """(query, leaf) tests per probe query against version v's tree."""
        ddm.ddm_attach(self.probe_ctx, self.ctx[v])
        ddm.ddm_plan(self.probe_ctx, self.probe[0], self.probe[1], stream=self.stream)
        return ddm.ddm_plan_stats(self.probe_ctx) / self.probe[0].shape[1]

    def acquire(self):
        with self.cv:
            v = self.active
            self.refs[v] += 1
            return v, self.step_of[v]

    def release(self, v):
        with self.cv:
            self.refs[v] -= 1
            self.cv.notify_all()

    def step(self, lo, hi, step_index: int):
        """Bring the idle version to the new coordinates (refit or rebuild)
        and activate it."""
        import torch
        with self.cv:
            idle = 1 - self.active
            while self.refs[idle]:
                self.cv.wait()
            self.stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(self.stream):
                self.pos[idle][0].copy_(lo)
                self.pos[idle][1].copy_(hi)
                if self.rebuild_every and step_index % self.rebuild_every == 0:
                    ddm.ddm_build(self.ctx[idle], self.pos[idle][0], self.pos[idle][1],
                                  stream=self.stream)
                    self.rebuilds += 1
                else:
                    ddm.ddm_refit(self.ctx[idle], self.pos[idle][0], self.pos[idle][1],
                                  stream=self.stream)
                    self.refits += 1
                    if self.probe_ctx is not None:
                        ratio = self._probe(idle) / max(self.base_tests[idle], 1e-9)
                        self.tests_ratio.append(ratio)
                        if ratio > self.adaptive:
                            ddm.ddm_build(self.ctx[idle], self.pos[idle][0], self.pos[idle][1],
                                          stream=self.stream)
                            self.rebuilds += 1
                            self.base_tests[idle] = self._probe(idle)
            self.step_of[idle] = step_index
            self.active = idle
            if self.history is not None:
                self.history[step_index] = (lo.clone(), hi.clone())

    def close(self):
        for c in self.ctx:
            ddm.ddm_destroy(c)
        if self.probe_ctx is not None:
            ddm.ddm_destroy(self.probe_ctx)
            self.probe_ctx = None


@dataclass
class Request:
    rid: int
    federate: int
    arrival: float          # seconds after the start
    size: int
    seed: int
    est_bytes: int = 0
    admitted: float = 0.0
    done: float = 0.0
    version: int = -1
    step: int = -1
    K: int = 0
    pairs: Optional[np.ndarray] = None
    lo: Any = None          # update set already on the device, (d, size); None: drawn
    hi: Any = None          # from `seed` when the request is admitted
    batch: int = -1         # launch the request ran in
    base: int = 0           # its first update id within that launch
    est_pairs: float = 0.0


def poisson_schedule(rate: float, duration: float, federates: int, size_lo: int, size_hi: int,
                     seed: int) -> List[Request]:
    """Requests of `federates` sources, Poisson in total at `rate` per second
    over `duration` seconds; sizes log-uniform in [size_lo, size_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        size = int(math.floor(math.exp(rng.uniform(math.log(size_lo), math.log(size_hi)))))
        out.append(Request(rid=len(out), federate=int(rng.integers(0, federates)), arrival=t,
                           size=size, seed=int(rng.integers(1, 2 ** 62))))
    return out


class Server:
    """Continuous batching of match requests under a device-memory budget.

    One dispatcher thread admits arrived requests in arrival order.  Whenever
    one of the `slots` (a context, a CUDA stream, staging and pair buffers)
    is free, every waiting request that fits the slot's limits and the memory
    budget is admitted into it at once: their update sets are concatenated
    and matched against the resident tree in ONE plan and ONE write pass
    (``ddm_plan_async`` / ``ddm_write_async``, no host synchronisation), and
    ``ddm_pair_offsets_async`` locates each request's pairs in the output,
    which is laid out by update id.  The launch pins the subscription version
    active at admission.  Slots run concurrently on their own streams; the
    dispatcher polls their events, so requests that arrive while others are
    on the GPU join the next free slot without waiting for them.  Under light
    load a launch holds one request (low latency); under heavy load launches
    grow (throughput).

    A request's pairs carry update ids relative to its own set: the pairs of
    a launch hold ids within the launch, and request r's slice is shifted by
    its base id ``r.base`` (done when ``keep_pairs`` copies them out)."""

    def __init__(self, regions: ResidentRegions, l: float, slots: int = 4,
                 budget_bytes: Optional[int] = None, pair_capacity: int = 1 << 25,
                 max_batch_updates: int = 1 << 24, max_batch_requests: int = 1024,
                 keep_pairs: bool = False):
        import torch
        self.regions = regions
        self.l = l
        self.keep_pairs = keep_pairs
        free, _ = torch.cuda.mem_get_info()
        self.budget = budget_bytes if budget_bytes is not None else int(free * 0.5)
        self.reserved = 0
        self.cap = pair_capacity
        self.max_updates = max_batch_updates
        self.max_requests = max_batch_requests
        d = regions.d
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                "ctx": ddm.ddm_create(torch.cuda.current_device()),
                "stream": torch.cuda.Stream(),
                "lo": torch.empty(d * max_batch_updates, dtype=torch.float32, device="cuda"),
                "hi": torch.empty(d * max_batch_updates, dtype=torch.float32, device="cuda"),
                "buf": torch.empty((pair_capacity, 2), dtype=torch.int32, device="cuda"),
                "uoff_h": torch.zeros(max_batch_requests + 1, dtype=torch.int64).pin_memory(),
                "uoff_d": torch.zeros(max_batch_requests + 1, dtype=torch.int64, device="cuda"),
                "poff_d": torch.zeros(max_batch_requests + 1, dtype=torch.int64, device="cuda"),
                "poff_h": torch.zeros(max_batch_requests + 1, dtype=torch.int64).pin_memory(),
                "kd": torch.zeros(1, dtype=torch.int64, device="cuda"),
                "ed": torch.zeros(1, dtype=torch.int32, device="cuda"),
                "kh": torch.zeros(1, dtype=torch.int64).pin_memory(),
                "eh": torch.zeros(1, dtype=torch.int32).pin_memory(),
                "event": torch.cuda.Event(),
                "batch": None, "ver": -1, "sets": None})
        self.t0 = 0.0
        self.launches = 0

    def expected_pairs(self, r: Request) -> float:
        # uniform placement: per dimension an update overlaps a region with
        # probability p = 2l/W - (l/W)^2 (W = L - l); E[K] = size * n * p^d
        W = L - self.l
        p = 2 * self.l / W - (self.l / W) ** 2
        return r.size * self.regions.n * p ** self.regions.d

    def estimate(self, r: Request) -> int:
        """Device bytes a request occupies while it runs: its share of a
        plan's workspace (sort, sorted copy, counts, offsets, records) and of
        the pair buffer."""
        r.est_pairs = self.expected_pairs(r)
        return int(r.size * (72 + 16 * self.regions.d) + 16 * r.est_pairs)

    def _launch(self, slot, batch: List[Request]):
        import torch
        v, step = self.regions.acquire()
        ctx, s, d = slot["ctx"], slot["stream"], self.regions.d
        ddm.ddm_attach(ctx, self.regions.ctx[v])
        sizes = np.array([r.size for r in batch], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(sizes)])
        M, count = int(offs[-1]), len(batch)
        with torch.cuda.stream(s):
            for r in batch:
                if r.lo is None:
                    r.lo, r.hi = request_updates(r.seed, r.size, d, self.l)
            if count == 1:
                lo, hi = batch[0].lo, batch[0].hi
            else:
                lo = slot["lo"][:d * M].view(d, M)
                hi = slot["hi"][:d * M].view(d, M)
                torch.cat([r.lo for r in batch], dim=1, out=lo)
                torch.cat([r.hi for r in batch], dim=1, out=hi)
            slot["uoff_h"][:count + 1].numpy()[:] = offs
            uoff = slot["uoff_d"][:count + 1]
            poff = slot["poff_d"][:count + 1]
            uoff.copy_(slot["uoff_h"][:count + 1], non_blocking=True)
            ddm.ddm_plan_async(ctx, lo, hi, stream=s)
            ddm.ddm_write_async(ctx, 0, M, slot["buf"], slot["kd"], slot["ed"], stream=s)
            ddm.ddm_pair_offsets_async(ctx, uoff, poff, stream=s)
            slot["kh"].copy_(slot["kd"], non_blocking=True)
            slot["eh"].copy_(slot["ed"], non_blocking=True)
            slot["poff_h"][:count + 1].copy_(poff, non_blocking=True)
            slot["event"].record(s)
        for i, r in enumerate(batch):
            r.version, r.step, r.batch, r.base = v, step, self.launches, int(offs[i])
        self.launches += 1
        slot["batch"], slot["ver"], slot["sets"] = batch, v, (lo, hi)

    def _alone(self, slot, r: Request):
        """One request by itself, its pairs streamed out in ordered chunks of
        the slot buffer (used when a launch's pairs overflow the buffer)."""
        import torch
        ctx, s = slot["ctx"], slot["stream"]
        with torch.cuda.stream(s):
            r.K = ddm.ddm_plan(ctx, r.lo, r.hi, stream=s)
            parts, b = [], 0
            while b < r.size:
                e = ddm.ddm_chunk_end_ordered(ctx, b, self.cap, stream=s)
                k = ddm.ddm_write_ordered(ctx, b, e, slot["buf"], stream=s)
                if self.keep_pairs:
                    parts.append(slot["buf"][:k].cpu().numpy().view(np.uint32).copy())
                b = e
        if self.keep_pairs:
            r.pairs = np.concatenate(parts) if parts else np.zeros((0, 2), np.uint32)
        r.base = 0

    def _finish(self, slot):
        batch = slot["batch"]
        err = int(slot["eh"][0])
        if err & 3:
            raise RuntimeError(f"launch of requests {[r.rid for r in batch]}: device error bits {err}")
        if err & 4:  # more pairs than the slot buffer: each request alone, chunked
            for r in batch:
                self._alone(slot, r)
        else:
            poff = slot["poff_h"][:len(batch) + 1].numpy().copy()
            host = None
            if self.keep_pairs and int(poff[-1]):
                host = slot["buf"][:int(poff[-1])].cpu().numpy().view(np.uint32)
            for i, r in enumerate(batch):
                r.K = int(poff[i + 1] - poff[i])
                if self.keep_pairs:
                    pr = (host[poff[i]:poff[i + 1]].copy() if host is not None
                          else np.zeros((0, 2), np.uint32))
                    pr[:, 0] -= np.uint32(r.base)
                    r.pairs = pr
        self.regions.release(slot["ver"])
        now = time.perf_counter() - self.t0
        for r in batch:
            r.done = now
            self.reserved -= r.est_bytes
            r.lo = r.hi = None
        slot["batch"], slot["sets"] = None, None

    def warm_up(self, size: Optional[int] = None, rounds: int = 2):
        """`rounds` launches of `size` updates per slot (default: the largest
        launch the slot limits allow), so that each slot's workspace and
        record arena are sized before serving (the library grows buffers with
        synchronous allocations)."""
        if size is None:
            per_update = self.expected_pairs(Request(0, 0, 0.0, 1, 0))
            size = min(self.max_updates, int(0.7 * self.cap / max(per_update, 1e-9)))
        for k in range(rounds):
            for i, slot in enumerate(self.slots):
                r = Request(rid=-1 - i, federate=0, arrival=0.0, size=size, seed=12345 + 97 * k + i)
                r.est_bytes = 0
                self._launch(slot, [r])
            for slot in self.slots:
                slot["event"].synchronize()
                self._finish(slot)
        self.launches = 0

    def run(self, schedule: List[Request], mover=None, step_s: float = 0.010,
            timeout_s: float = 600.0) -> List[Request]:
        """Serve `schedule` in real time; `mover(step)` returns the regions'
        coordinates after movement step `step`; a separate thread applies a
        step every step_s (refit of the idle version), so admissions never
        wait for a refit."""
        self.t0 = time.perf_counter()
        stop = threading.Event()

        def move():
            import torch
            step, next_step = 0, step_s
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                while not stop.is_set():
                    now = time.perf_counter() - self.t0
                    if now < next_step:
                        time.sleep(min(0.001, next_step - now))
                        continue
                    step += 1
                    lo, hi = mover(step)
                    self.regions.step(lo, hi, step)
                    next_step += step_s

        mover_thread = threading.Thread(target=move, daemon=True) if mover is not None else None
        if mover_thread:
            mover_thread.start()
        try:
            return self._serve(schedule, timeout_s)
        finally:
            stop.set()
            if mover_thread:
                mover_thread.join()

    def _take(self) -> List[Request]:
        """The next launch: waiting requests in arrival order while they fit
        the slot (updates, requests, expected pairs) and the memory budget."""
        batch, M, pairs = [], 0, 0.0
        while self.waiting and len(batch) < self.max_requests:
            r = self.waiting[0]
            if not r.est_bytes:
                r.est_bytes = self.estimate(r)
            if batch and (M + r.size > self.max_updates or pairs + r.est_pairs > 0.7 * self.cap):
                break
            if (batch or self.reserved) and self.reserved + r.est_bytes > self.budget:
                break
            self.waiting.popleft()
            self.reserved += r.est_bytes
            r.admitted = time.perf_counter() - self.t0
            batch.append(r)
            M += r.size
            pairs += r.est_pairs
        return batch

    def _serve(self, schedule, timeout_s):
        pending = deque(sorted(schedule, key=lambda r: r.arrival))
        self.waiting: Deque[Request] = deque()
        finished: List[Request] = []
        while len(finished) < len(schedule):
            now = time.perf_counter() - self.t0
            if now > timeout_s:
                raise TimeoutError("serving run did not finish")
            while pending and pending[0].arrival <= now:
                self.waiting.append(pending.popleft())
            for slot in self.slots:  # completions
                if slot["batch"] is not None and slot["event"].query():
                    finished.extend(slot["batch"])
                    self._finish(slot)
            for slot in self.slots:  # admissions
                if not self.waiting:
                    break
                if slot["batch"] is None:
                    batch = self._take()
                    if not batch:
                        break
                    self._launch(slot, batch)
            if all(sl["batch"] is not None for sl in self.slots) or not self.waiting:
                time.sleep(0.00005)
        return sorted(finished, key=lambda r: r.rid)

    def close(self):
        for sl in self.slots:
            ddm.ddm_destroy(sl["ctx"])


def summary(reqs: List[Request], wall: float) -> Dict[str, float]:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    K = sum(r.K for r in reqs)
    q = sum(r.size for r in reqs)
    return {"requests": len(reqs), "wall_s": wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "pairs": K, "pairs_per_s": K / wall,
            "queries_per_s": q / wall, "requests_per_s": len(reqs) / wall}
