"""Host logic of the serving loop on CPU: admission of waiting requests into a
launch (arrival order, the slot's limits, the memory budget), the request
size estimate and the Poisson schedule.  No GPU is used: the server is built
without its device buffers, since admission only reads sizes and estimates."""
import math
import time
from collections import deque

import numpy as np
import pytest

from paper_1309_3458_gb300 import serving as S


class _Regions:
    def __init__(self, n, d):
        self.n, self.d = n, d


def _server(n=1_000_000, d=2, l=1e3, cap=1 << 20, max_updates=1 << 16, max_requests=8,
            budget=1 << 40):
    srv = object.__new__(S.Server)   # admission needs no device state
    srv.regions = _Regions(n, d)
    srv.l = l
    srv.cap = cap
    srv.max_updates = max_updates
    srv.max_requests = max_requests
    srv.budget = budget
    srv.reserved = 0
    srv.t0 = time.perf_counter()
    srv.waiting = deque()
    return srv


def _req(rid, size):
    return S.Request(rid=rid, federate=0, arrival=0.0, size=size, seed=rid + 1)


def test_overlap_probability_closed_form():
    """p = 2l/W - (l/W)^2 is the chance that two closed segments of length l
    with lower bounds uniform in [0, W] overlap; Monte Carlo agrees."""
    srv = _server(n=1, d=1, l=2e5)
    p = srv.expected_pairs(_req(0, 1))
    W = S.L - srv.l
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, W, 1_000_000), rng.uniform(0, W, 1_000_000)
    mc = np.mean(np.abs(x - y) <= srv.l)
    assert abs(mc - p) < 4 * math.sqrt(p * (1 - p) / 1_000_000)
    # d dimensions, n regions, size updates: size * n * p^d
    srv2 = _server(n=1000, d=2, l=2e5)
    assert srv2.expected_pairs(_req(0, 10)) == pytest.approx(10 * 1000 * p ** 2)


def test_take_admits_in_arrival_order_within_limits():
    srv = _server(max_requests=3)
    reqs = [_req(i, 100) for i in range(5)]
    srv.waiting.extend(reqs)
    batch = srv._take()
    assert [r.rid for r in batch] == [0, 1, 2]              # request limit, FIFO
    assert [r.rid for r in srv.waiting] == [3, 4]
    assert srv.reserved == sum(r.est_bytes for r in batch) > 0
    assert all(r.est_bytes == srv.estimate(r) for r in batch)


def test_take_stops_at_the_update_and_pair_limits():
    srv = _server(max_updates=1000, max_requests=100)
    srv.waiting.extend([_req(0, 600), _req(1, 300), _req(2, 200), _req(3, 1)])
    assert [r.rid for r in srv._take()] == [0, 1]           # 600 + 300 <= 1000 < 1100
    # no skipping: request 3 would fit but waits behind request 2
    assert [r.rid for r in srv.waiting] == [2, 3]
    # pair limit: 0.7 of the slot's pair buffer by expected pairs
    srv2 = _server(max_updates=1 << 30, max_requests=100)
    per = srv2.expected_pairs(_req(0, 1))
    size = int(0.3 * srv2.cap / per)
    srv2.waiting.extend([_req(i, size) for i in range(4)])
    assert len(srv2._take()) == 2                            # 0.6 cap fits, 0.9 does not


def test_take_budget_and_no_starvation():
    srv = _server(budget=10_000_000)
    big = _req(0, 1_000_000)                                 # alone above the budget
    srv.waiting.extend([big, _req(1, 10)])
    batch = srv._take()
    assert batch == [big]       # nothing reserved: the head is admitted anyway
    assert srv._take() == []    # the budget is now exceeded: the next one waits
    srv.reserved -= big.est_bytes
    assert [r.rid for r in srv._take()] == [1]


def test_poisson_schedule():
    a = S.poisson_schedule(2000.0, 2.0, 64, 1000, 1_000_000, seed=5)
    b = S.poisson_schedule(2000.0, 2.0, 64, 1000, 1_000_000, seed=5)
    assert [(r.arrival, r.size, r.seed) for r in a] == [(r.arrival, r.size, r.seed) for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    assert abs(len(a) - 4000) < 4 * math.sqrt(4000)         # Poisson count
    sizes = np.array([r.size for r in a])
    assert sizes.min() >= 1000 and sizes.max() <= 1_000_000
    # log-uniform: the median is near the geometric mean of the bounds
    assert abs(math.log(np.median(sizes)) - math.log(math.sqrt(1000 * 1e6))) < 0.3
    assert {r.federate for r in a} <= set(range(64))
