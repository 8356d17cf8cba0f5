"""Host logic of the serving loop (no GPU): the request workload, Poisson arrivals, batch admission
(slots, points and HBM budget, scenes not yet resident, failed scenes) and the latency summary."""
import collections
import math
import threading

import numpy as np

from paper_2504_19163_gb300 import scenes as S
from paper_2504_19163_gb300 import serving as SV


def test_workload_mix_is_seeded_and_in_range():
    a = SV.make_requests(512, seed=5)
    b = SV.make_requests(512, seed=5)
    assert [(r.scene, r.emitters, r.n_side, r.seed) for r in a] == [(r.scene, r.emitters, r.n_side, r.seed) for r in b]
    assert {r.scene for r in a} == set(S.SERVING_SCENES)
    assert {r.n_side for r in a} == set(SV.SIDES)
    for r in a:
        assert 1 <= len(r.emitters) <= S.SERVING_POOL
        assert list(r.emitters) == sorted(set(r.emitters))
        assert all(0 <= e < S.SERVING_POOL for e in r.emitters)
    sizes = collections.Counter(len(r.emitters) for r in a)
    assert len(sizes) == S.SERVING_POOL  # every subset size occurs


def test_poisson_arrivals_rate():
    reqs = SV.make_requests(20000, seed=1, sides=(64,))
    SV.poisson_arrivals(reqs, rate=50.0, seed=2)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # mean gap 1/rate within 5 standard errors; exponential: sd = mean
    assert abs(gaps.mean() - 1 / 50.0) < 5 * (1 / 50.0) / math.sqrt(gaps.size)
    # memoryless: P(gap > mean) = e^-1
    assert abs(np.mean(gaps > 1 / 50.0) - math.exp(-1)) < 0.02


class FakeEntry:
    def __init__(self, ready=True, error=None):
        self.ready = threading.Event()
        if ready:
            self.ready.set()
        self.error = error
        self.in_flight = 0
        self.resident = None


class FakeCache:
    def __init__(self, entries):
        self.entries = entries
        self.lock = threading.Lock()

    def request(self, name):
        return self.entries[name]


def fake_server(entries, max_jobs, max_points, hbm_budget, in_flight_bytes=0):
    srv = object.__new__(SV.Server)
    srv.cache = FakeCache(entries)
    srv.max_jobs = max_jobs
    srv.max_points = max_points
    srv.hbm_budget = hbm_budget
    srv.in_flight_bytes = in_flight_bytes
    return srv


def req(i, scene, side):
    return SV.Request(i, scene, (0,), side, i)


def test_admission_respects_slots_points_and_arrival_order():
    entries = {"a": FakeEntry(), "b": FakeEntry(ready=False), "c": FakeEntry(error=RuntimeError("x"))}
    srv = fake_server(entries, max_jobs=3, max_points=3 * 128 * 128, hbm_budget=1 << 40)
    pending = collections.deque([req(0, "b", 64), req(1, "a", 128), req(2, "c", 64), req(3, "a", 64),
                                 req(4, "a", 128), req(5, "a", 64), req(6, "a", 64)])
    batch, failed = srv._form_batch(pending, 0.0)
    # b is not resident yet (kept, first in line); c failed to build; a's requests fill 3 slots
    assert [r.rid for r in batch] == [1, 3, 4]
    assert [r.rid for r in failed] == [2] and failed[0].status != 0
    assert [r.rid for r in pending] == [0, 5, 6]
    assert entries["a"].in_flight == 3
    # points limit: the first request that does not fit stops the batch (no overtaking)
    srv2 = fake_server({"a": FakeEntry()}, max_jobs=8, max_points=128 * 128 + 64 * 64, hbm_budget=1 << 40)
    pending = collections.deque([req(0, "a", 128), req(1, "a", 128), req(2, "a", 64)])
    batch, _ = srv2._form_batch(pending, 0.0)
    assert [r.rid for r in batch] == [0]
    assert [r.rid for r in pending] == [1, 2]


def test_admission_respects_the_hbm_budget():
    e = {"a": FakeEntry()}
    per = SV.Server.request_bytes(req(0, "a", 256))
    srv = fake_server(e, max_jobs=8, max_points=1 << 30, hbm_budget=3 * per, in_flight_bytes=per)
    pending = collections.deque([req(i, "a", 256) for i in range(5)])
    batch, _ = srv._form_batch(pending, 0.0)
    assert len(batch) == 2 and len(pending) == 3
    srv.in_flight_bytes = 3 * per  # budget full: nothing admitted until a batch completes
    batch, _ = srv._form_batch(pending, 0.0)
    assert batch == [] and len(pending) == 3


def test_summary_percentiles():
    reqs = [req(i, "a", 64) for i in range(100)]
    for i, r in enumerate(reqs):
        r.arrival = float(i)
        r.t_done = float(i) + (i + 1) * 1e-3
        r.E = np.zeros(1, np.float32)
    s = SV.summarize(reqs)
    assert s["completed"] == 100
    assert abs(s["p50_ms"] - 50.5) < 1e-6
    assert abs(s["p99_ms"] - np.percentile(np.arange(1, 101), 99)) < 1e-6
    assert abs(s["samples_per_s"] - 100 * 64 * 64 / (99 + 0.1)) < 1e-6


def test_pooled_traces_take_percentiles_over_all_latencies():
    a = {"requests": 100, "completed": 100, "p50_ms": 0.0, "p99_ms": 0.0, "mean_ms": 0.0, "samples_per_s": 10.0,
         "requests_per_s": 1.0, "span_s": 1.0, "_lat": np.linspace(0.001, 0.100, 100)}
    b = dict(a, samples_per_s=30.0, _lat=np.linspace(0.101, 0.200, 100))
    p = SV.pooled([a, b])
    lat = np.concatenate([a["_lat"], b["_lat"]])
    assert p["traces"] == 2 and p["requests"] == 200 and p["completed"] == 200
    assert abs(p["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
    assert abs(p["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert p["samples_per_s"] == 20.0
    assert "_lat" not in SV.pooled([a])
