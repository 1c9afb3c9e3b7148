"""Serving loop: continuous batching of match requests against resident,
moving subscription regions.

The paper's dynamic setting (Section IV, "Dynamic interval management"):
extents move, and each update set queries the subscription tree again.  Here
the subscriptions stay resident on the device in two tree versions; every
movement step refits the idle version in place (``ddm_refit``: same order,
new per-node bounds) and makes it the active one.  Match requests (update
sets of any size) arrive over time; each is admitted to a free slot when the
memory budget allows, pins the version active at admission, and runs on the
slot's own CUDA stream and context (``ddm_attach``), so requests admitted
while others run overlap on the GPU.  A version is refitted only when no
request pins it, so a request's result does not depend on what else runs.

Host orchestration only: every step of the matching runs in libddm's
kernels.  Update sets and movement are synthesised on the device with seeded
torch generators (workload generation, not matching arithmetic).
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

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
    """Subscriptions kept on the device in two tree versions."""

    def __init__(self, lo, hi, keep_history: bool = False):
        import torch
        self.d, self.n = lo.shape
        self.ctx = [ddm.ddm_create(lo.device.index or 0) for _ in range(2)]
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
        """Refit the idle version to the new coordinates and activate it."""
        import torch
        with self.cv:
            idle = 1 - self.active
            while self.refs[idle]:
                self.cv.wait()
            self.stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(self.stream):
                self.pos[idle][0].copy_(lo)
                self.pos[idle][1].copy_(hi)
                ddm.ddm_refit(self.ctx[idle], self.pos[idle][0], self.pos[idle][1],
                              stream=self.stream)
            self.step_of[idle] = step_index
            self.active = idle
            if self.history is not None:
                self.history[step_index] = (lo.clone(), hi.clone())

    def close(self):
        for c in self.ctx:
            ddm.ddm_destroy(c)


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
    """Continuous batching over `slots` contexts, each with its own CUDA
    stream, under a device-memory budget.

    One dispatcher thread admits arrived requests into free slots (arrival
    order, while the budget allows), enqueues each request's whole match with
    the host-synchronisation-free calls (generation of its update set,
    ``ddm_plan_async``, ``ddm_write_async``, an event), and polls the slots'
    events; requests therefore overlap on the GPU without waiting for one
    another.  A request pins the subscription version active when it is
    admitted and releases it when its event completes."""

    def __init__(self, regions: ResidentRegions, l: float, slots: int = 8,
                 budget_bytes: Optional[int] = None, pair_capacity: int = 1 << 25,
                 keep_pairs: bool = False):
        import torch
        self.regions = regions
        self.l = l
        self.keep_pairs = keep_pairs
        free, _ = torch.cuda.mem_get_info()
        self.budget = budget_bytes if budget_bytes is not None else int(free * 0.5)
        self.reserved = 0
        self.cap = pair_capacity
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                "ctx": ddm.ddm_create(torch.cuda.current_device()),
                "stream": torch.cuda.Stream(),
                "buf": torch.empty((pair_capacity, 2), dtype=torch.int32, device="cuda"),
                "kd": torch.zeros(1, dtype=torch.int64, device="cuda"),
                "ed": torch.zeros(1, dtype=torch.int32, device="cuda"),
                "kh": torch.zeros(1, dtype=torch.int64).pin_memory(),
                "eh": torch.zeros(1, dtype=torch.int32).pin_memory(),
                "event": torch.cuda.Event(),
                "req": None, "ver": -1, "keep": None})
        self.t0 = 0.0

    def estimate(self, r: Request) -> int:
        # workspace of one plan (sort, sorted copy, counts, offsets, records)
        # plus the expected pairs: E[K] = m * n * p^d, p = 2l/W - (l/W)^2
        W = L - self.l
        p = 2 * self.l / W - (self.l / W) ** 2
        k = r.size * self.regions.n * p ** self.regions.d
        return int(r.size * (72 + 16 * self.regions.d) + 16 * k)

    def _launch(self, slot, r: Request):
        import torch
        v, step = self.regions.acquire()
        ctx, s = slot["ctx"], slot["stream"]
        ddm.ddm_attach(ctx, self.regions.ctx[v])
        with torch.cuda.stream(s):
            lo, hi = request_updates(r.seed, r.size, self.regions.d, self.l)
            ddm.ddm_plan_async(ctx, lo, hi, stream=s)
            ddm.ddm_write_async(ctx, 0, r.size, slot["buf"], slot["kd"], slot["ed"], stream=s)
            slot["kh"].copy_(slot["kd"], non_blocking=True)
            slot["eh"].copy_(slot["ed"], non_blocking=True)
            slot["event"].record(s)
        slot["req"], slot["ver"], slot["keep"] = r, v, (lo, hi)
        r.version, r.step = v, step

    def _finish(self, slot):
        import torch
        r = slot["req"]
        err = int(slot["eh"][0])
        if err & 1:
            raise ValueError(f"request {r.rid}: invalid extent")
        if err & 4:  # more pairs than the slot buffer: stream them out in ordered chunks
            ctx, s = slot["ctx"], slot["stream"]
            with torch.cuda.stream(s):
                lo, hi = slot["keep"]
                r.K = ddm.ddm_plan(ctx, lo, hi, stream=s)
                parts, b = [], 0
                while b < r.size:
                    e = ddm.ddm_chunk_end_ordered(ctx, b, self.cap, stream=s)
                    k = ddm.ddm_write_ordered(ctx, b, e, slot["buf"], stream=s)
                    if self.keep_pairs:
                        parts.append(slot["buf"][:k].cpu().numpy().view(np.uint32).copy())
                    b = e
                if self.keep_pairs:
                    r.pairs = np.concatenate(parts) if parts else np.zeros((0, 2), np.uint32)
        else:
            r.K = int(slot["kh"][0])
            if self.keep_pairs:
                with torch.cuda.stream(slot["stream"]):
                    r.pairs = slot["buf"][:r.K].cpu().numpy().view(np.uint32).copy()
        self.regions.release(slot["ver"])
        r.done = time.perf_counter() - self.t0
        self.reserved -= r.est_bytes
        slot["req"], slot["keep"] = None, None

    def warm_up(self, size: int):
        """One request of `size` updates per slot, so that each slot's
        workspace and record arena are sized before serving (the library
        grows buffers with synchronous allocations)."""
        for i, slot in enumerate(self.slots):
            r = Request(rid=-1 - i, federate=0, arrival=0.0, size=size, seed=12345 + i)
            self._launch(slot, r)
        for slot in self.slots:
            slot["event"].synchronize()
            self._finish(slot)
        # a second round, now that each context knows its record arena size
        for i, slot in enumerate(self.slots):
            self._launch(slot, Request(rid=-1 - i, federate=0, arrival=0.0, size=size,
                                       seed=54321 + i))
        for slot in self.slots:
            slot["event"].synchronize()
            self._finish(slot)

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

    def _serve(self, schedule, timeout_s):
        pending = list(schedule)
        waiting: List[Request] = []
        finished: List[Request] = []
        while len(finished) < len(schedule):
            now = time.perf_counter() - self.t0
            if now > timeout_s:
                raise TimeoutError("serving run did not finish")
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            for slot in self.slots:  # completions
                if slot["req"] is not None and slot["event"].query():
                    r = slot["req"]
                    self._finish(slot)
                    finished.append(r)
            for slot in self.slots:  # admissions, in arrival order
                if not waiting:
                    break
                if slot["req"] is not None:
                    continue
                r = waiting[0]
                r.est_bytes = self.estimate(r)
                if self.reserved and self.reserved + r.est_bytes > self.budget:
                    break
                waiting.pop(0)
                self.reserved += r.est_bytes
                r.admitted = time.perf_counter() - self.t0
                self._launch(slot, r)
            if all(sl["req"] is not None for sl in self.slots) or not waiting:
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
