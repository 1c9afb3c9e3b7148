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
import queue
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
    """Continuous batching over `slots` contexts/streams with a byte budget."""

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
        self.lock = threading.Lock()
        self.cap = pair_capacity
        self.slots = []
        for _ in range(slots):
            ctx = ddm.ddm_create(torch.cuda.current_device())
            s = torch.cuda.Stream()
            buf = torch.empty((pair_capacity, 2), dtype=torch.int32, device="cuda")
            inbox: "queue.Queue[Optional[Request]]" = queue.Queue()
            self.slots.append({"ctx": ctx, "stream": s, "buf": buf, "inbox": inbox, "busy": False})
        self.done: "queue.Queue[Request]" = queue.Queue()
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for t in self.threads:
            t.start()
        self.t0 = 0.0

    def estimate(self, r: Request) -> int:
        # workspace of one plan (sort, sorted copy, counts, offsets, records)
        # plus the expected pairs: E[K] = m * n * p^d, p = 2l/W - (l/W)^2
        W = L - self.l
        p = 2 * self.l / W - (self.l / W) ** 2
        k = r.size * self.regions.n * p ** self.regions.d
        return int(r.size * (72 + 16 * self.regions.d) + 16 * k)

    def _worker(self, i: int):
        import torch
        slot = self.slots[i]
        ctx, s, buf = slot["ctx"], slot["stream"], slot["buf"]
        while True:
            r = slot["inbox"].get()
            if r is None:
                return
            v, step = self.regions.acquire()
            try:
                ddm.ddm_attach(ctx, self.regions.ctx[v])
                with torch.cuda.stream(s):
                    lo, hi = request_updates(r.seed, r.size, self.regions.d, self.l)
                    r.K = ddm.ddm_plan(ctx, lo, hi, stream=s)
                    parts = []
                    b = 0
                    while b < r.size:
                        e = ddm.ddm_chunk_end_ordered(ctx, b, self.cap, stream=s)
                        k = ddm.ddm_write_ordered(ctx, b, e, buf, stream=s)
                        if self.keep_pairs:
                            parts.append(buf[:k].cpu().numpy().view(np.uint32).copy())
                        b = e
                    if self.keep_pairs:
                        r.pairs = np.concatenate(parts) if parts else np.zeros((0, 2), np.uint32)
                    s.synchronize()
            finally:
                self.regions.release(v)
            r.version, r.step = v, step
            r.done = time.perf_counter() - self.t0
            with self.lock:
                self.reserved -= r.est_bytes
                slot["busy"] = False
            self.done.put(r)

    def run(self, schedule: List[Request], mover=None, step_s: float = 0.010,
            timeout_s: float = 600.0) -> List[Request]:
        """Serve `schedule` in real time; `mover(step)` returns the regions'
        coordinates after movement step `step` (called every step_s)."""
        pending = list(schedule)
        waiting: List[Request] = []
        finished: List[Request] = []
        self.t0 = time.perf_counter()
        next_step, step = step_s, 0
        while len(finished) < len(schedule):
            now = time.perf_counter() - self.t0
            if now > timeout_s:
                raise TimeoutError("serving run did not finish")
            if mover is not None and now >= next_step:
                step += 1
                lo, hi = mover(step)
                self.regions.step(lo, hi, step)
                next_step += step_s
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # admit in arrival order while a slot is free and the budget allows
            while waiting:
                r = waiting[0]
                r.est_bytes = self.estimate(r)
                with self.lock:
                    free = [i for i, sl in enumerate(self.slots) if not sl["busy"]]
                    fits = self.reserved + r.est_bytes <= self.budget or self.reserved == 0
                    if not free or not fits:
                        break
                    self.reserved += r.est_bytes
                    self.slots[free[0]]["busy"] = True
                waiting.pop(0)
                r.admitted = time.perf_counter() - self.t0
                self.slots[free[0]]["inbox"].put(r)
            try:
                while True:
                    finished.append(self.done.get_nowait())
            except queue.Empty:
                pass
            time.sleep(0.0001)
        return sorted(finished, key=lambda r: r.rid)

    def close(self):
        for sl in self.slots:
            sl["inbox"].put(None)
        for t in self.threads:
            t.join()
        for sl in self.slots:
            ddm.ddm_destroy(sl["ctx"])


def summary(reqs: List[Request], wall: float) -> Dict[str, float]:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    K = sum(r.K for r in reqs)
    q = sum(r.size for r in reqs)
    return {"requests": len(reqs), "wall_s": wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "pairs": K, "pairs_per_s": K / wall,
            "queries_per_s": q / wall, "requests_per_s": len(reqs) / wall}
