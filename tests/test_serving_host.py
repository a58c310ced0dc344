"""Host logic of the serving loop (continuous batching, admission, latency
statistics) against a stand-in index: no GPU needed."""
import threading
import time

import numpy as np

from paper_2607_02543_gb300.serve import Request, Server, percentiles, poisson_stream, overlap_seconds


class FakeIndex:
    degree = 4

    def __init__(self, free=10_000):
        self.free0 = free
        self.free = free
        self.next = 100
        self.concurrent = False
        self.lock = threading.Lock()
        self.batches = []

    def set_concurrent(self, on):
        self.concurrent = on

    def search(self, q, k, beam, stream=None):
        time.sleep(0.003)
        with self.lock:
            self.batches.append(("query", len(q)))
        ids = np.tile(np.arange(k, dtype=np.uint32), (len(q), 1))
        return ids, np.zeros((len(q), k), np.float32) + q[:, :1]

    def insert(self, x, stream=None):
        time.sleep(0.002)
        with self.lock:
            self.free -= len(x) * (self.degree + 1)
            ids = np.arange(self.next, self.next + len(x), dtype=np.uint32)
            self.next += len(x)
            self.batches.append(("insert", len(x)))
        return ids

    def delete(self, ids, stream=None):
        with self.lock:
            self.batches.append(("delete", len(ids)))
        return len(ids)

    def reclaim(self, stream=None):
        with self.lock:
            self.free = self.free0
            self.batches.append(("reclaim", 0))

    def stats(self):
        return {"free_slabs": self.free, "live": self.next, "used_slabs": self.free0 - self.free}


def _requests(rng, n_q=200, n_u=40, dim=4, rate_q=4000.0, rate_u=800.0):
    tq = np.sort(rng.uniform(0, n_q / rate_q, n_q))
    tu = np.sort(rng.uniform(0, n_u / rate_u, n_u))
    reqs = [Request(float(t), "query", rng.normal(size=dim).astype(np.float32)) for t in tq]
    for i, t in enumerate(tu):
        if i % 2 == 0:
            reqs.append(Request(float(t), "insert", rng.normal(size=(3, dim)).astype(np.float32)))
        else:
            reqs.append(Request(float(t), "delete", np.array([i], np.uint32)))
    return sorted(reqs, key=lambda r: r.t)


def test_every_request_served_and_batched():
    rng = np.random.default_rng(0)
    reqs = _requests(rng)
    idx = FakeIndex()
    out = Server(idx, k=5, beam=8).run(reqs)
    assert all(np.isfinite(r.done) and r.done >= r.t for r in reqs)
    assert out["queries"]["n"] == 200 and out["updates"]["n"] == 40
    # arrivals faster than one search batch: later batches hold several requests
    qb = [n for kind, n in idx.batches if kind == "query"]
    assert sum(qb) == 200 and max(qb) > 1
    assert out["query_batches"] < 200
    # every query's result is its own row (the stand-in echoes q[0])
    for r in reqs:
        if r.kind == "query":
            assert r.result[1][0] == r.payload[0]
    assert not idx.concurrent          # switched off again after the run


def test_admission_reclaims_then_admits():
    rng = np.random.default_rng(1)
    reqs = _requests(rng, n_q=10, n_u=20)
    idx = FakeIndex(free=2 * 2 * 3 * (4 + 1) + 1)   # room for about one insert batch
    srv = Server(idx, k=5, beam=8)
    srv.run(reqs)
    assert srv.reclaims > 0
    assert all(np.isfinite(r.done) for r in reqs)


def test_percentiles_and_poisson():
    p = percentiles([0.001] * 99 + [0.1])
    assert abs(p["p50_ms"] - 1.0) < 1e-9 and p["p99_ms"] > 1.0
    assert percentiles([])["n"] == 0
    t = poisson_stream(np.random.default_rng(2), 1000.0, 2.0)
    assert 1800 < t.size < 2200 and (np.diff(t) >= 0).all()
    assert overlap_seconds([("query", 0.0, 1.0), ("update", 0.5, 2.0)]) == 0.5
