"""Serving loops: queries and updates over one index.

Updates run on their own CUDA stream in concurrent mode (include/etale.h,
etale_set_concurrent), so their kernels overlap the queries' on the device as
the paper's two-stream experiment does (Sec. 5.5).  The update worker admits
an insert batch only when the free slab pool covers its worst case;
otherwise it first reclaims (which returns tombstone slabs) and, if that is
not enough, defers the batch.

Queries are served in one of two ways:
- Server: a query worker forms its next batch from every request that has
  arrived while its previous batch ran, up to a size cap (batch-granular);
- RingServer: slot-granular.  Arriving queries are written into the slots of
  a serving ring (etale_ring_*) and published at once; one bounded persistent
  launch is always in flight, and its warps take each query as soon as one
  is free, including queries that arrived after the launch started.

Latency of a request = completion time - arrival time.
"""
from __future__ import annotations

import dataclasses
import math
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    t: float                  # arrival, seconds from the start of the run
    kind: str                 # "query", "insert" or "delete"
    payload: np.ndarray       # query rows, insert rows or delete ids
    done: float = math.nan    # completion, seconds from the start
    result: object = None     # query: (ids, dists); insert: new ids; delete: count
    issued: float = math.nan  # when the batch holding it was issued


def poisson_stream(rng: np.random.Generator, rate: float, duration: float) -> np.ndarray:
    """Arrival times of a Poisson process of `rate` per second on [0, duration)."""
    n = rng.poisson(rate * duration)
    return np.sort(rng.uniform(0.0, duration, size=n))


def percentiles(lat_s: list[float]) -> dict:
    if not lat_s:
        return {"n": 0, "p50_ms": None, "p99_ms": None, "mean_ms": None}
    a = np.asarray(lat_s) * 1e3
    return {"n": int(a.size), "p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean())}


class Server:
    """Continuous-batching request loop.

    index: an object with search(q, k, beam, stream), insert(x, stream),
    delete(ids, stream), reclaim(stream), stats(), set_concurrent(on) and a
    `degree` attribute (paper_2607_02543_gb300.Index, or a stand-in).
    """

    def __init__(self, index, k: int = 10, beam: int = 64, max_query_batch: int = 4096,
                 max_update_batch: int = 4096, streams=(None, None), reclaim_every: int = 0):
        self.index, self.k, self.beam = index, k, beam
        self.max_q, self.max_u = max_query_batch, max_update_batch
        self.qstream, self.ustream = streams
        self.reclaim_every = reclaim_every
        self.log: list[tuple] = []          # (worker, t_issue, t_done, kind, n)
        self.deferred = 0
        self.reclaims = 0
        self.stats_over_time: list[dict] = []

    # --- admission ---------------------------------------------------------
    def slabs_needed(self, kind: str, n: int) -> int:
        R = self.index.degree
        # worst case of one update call: every publication takes a fresh slab
        if kind == "insert":
            return 2 * n * (R + 1)
        if kind == "delete":
            return n * R
        return 0

    def admit(self, kind: str, n: int) -> bool:
        need = self.slabs_needed(kind, n)
        if need == 0:
            return True
        if self.index.stats()["free_slabs"] >= need:
            return True
        self.index.reclaim(self.ustream)
        self.reclaims += 1
        return self.index.stats()["free_slabs"] >= need

    # --- workers -----------------------------------------------------------
    def _pending(self, reqs, i, now, cap):
        j = i
        while j < len(reqs) and reqs[j].t <= now and j - i < cap:
            j += 1
        return j

    def _query_worker(self, reqs, t0):
        i = 0
        while i < len(reqs):
            now = time.perf_counter() - t0
            if reqs[i].t > now:
                time.sleep(min(reqs[i].t - now, 0.002))
                continue
            j = self._pending(reqs, i, now, self.max_q)
            batch = reqs[i:j]
            q = np.concatenate([r.payload.reshape(1, -1) for r in batch]).astype(np.float32)
            issued = time.perf_counter() - t0
            ids, dists = self.index.search(q, self.k, self.beam, self.qstream)
            done = time.perf_counter() - t0
            for r, a, b in zip(batch, ids, dists):
                r.result, r.done, r.issued = (a, b), done, issued
            self.log.append(("query", issued, done, "query", len(batch)))
            i = j

    def _update_worker(self, reqs, t0):
        i, calls = 0, 0
        while i < len(reqs):
            now = time.perf_counter() - t0
            if reqs[i].t > now:
                time.sleep(min(reqs[i].t - now, 0.002))
                continue
            # one batch = the longest run of same-kind requests that arrived
            kind = reqs[i].kind
            j = i
            n = 0
            while (j < len(reqs) and reqs[j].t <= now and reqs[j].kind == kind
                   and n + len(reqs[j].payload) <= self.max_u):
                n += len(reqs[j].payload)
                j += 1
            if j == i:
                j, n = i + 1, len(reqs[i].payload)
            batch = reqs[i:j]
            if not self.admit(kind, n):
                self.deferred += 1
                time.sleep(0.001)
                continue
            issued = time.perf_counter() - t0
            if kind == "insert":
                x = np.concatenate([r.payload for r in batch]).astype(np.float32)
                ids = self.index.insert(x, self.ustream)
                off = 0
                for r in batch:
                    r.result = ids[off:off + len(r.payload)]
                    off += len(r.payload)
            else:
                d = np.concatenate([r.payload for r in batch]).astype(np.uint32)
                cnt = self.index.delete(d, self.ustream)
                for r in batch:
                    r.result = cnt
            calls += 1
            if self.reclaim_every and calls % self.reclaim_every == 0:
                self.index.reclaim(self.ustream)
                self.reclaims += 1
            done = time.perf_counter() - t0
            for r in batch:
                r.done, r.issued = done, issued
            self.log.append(("update", issued, done, kind, n))
            st = self.index.stats()
            self.stats_over_time.append({"t": done, "live": st["live"], "used_slabs": st["used_slabs"],
                                         "free_slabs": st["free_slabs"]})
            i = j

    def run(self, requests: list[Request]) -> dict:
        """Serve the requests (sorted by arrival) and return latency statistics."""
        queries = [r for r in requests if r.kind == "query"]
        updates = [r for r in requests if r.kind != "query"]
        self.index.set_concurrent(True)
        t0 = time.perf_counter()
        tq = threading.Thread(target=self._query_worker, args=(queries, t0))
        tu = threading.Thread(target=self._update_worker, args=(updates, t0))
        tq.start()
        tu.start()
        tq.join()
        tu.join()
        wall = time.perf_counter() - t0
        self.index.set_concurrent(False)
        ql = [r.done - r.t for r in queries]
        ul = [r.done - r.t for r in updates]
        return {"wall_s": wall, "queries": percentiles(ql), "updates": percentiles(ul),
                "query_throughput": len(queries) / wall if wall > 0 else 0.0,
                "update_vectors_per_s": sum(len(r.payload) for r in updates) / wall if wall > 0 else 0.0,
                "query_batches": sum(1 for e in self.log if e[0] == "query"),
                "update_batches": sum(1 for e in self.log if e[0] == "update"),
                "deferred": self.deferred, "reclaims": self.reclaims}


def overlap_seconds(log) -> float:
    """Total time during which a query batch and an update batch were both in
    flight (from the host-side issue / completion times)."""
    q = [(a, b) for w, a, b, *_ in log if w == "query"]
    u = [(a, b) for w, a, b, *_ in log if w == "update"]
    tot = 0.0
    for qa, qb in q:
        for ua, ub in u:
            tot += max(0.0, min(qb, ub) - max(qa, ua))
    return tot


class RingServer(Server):
    """Slot-granular serving: queries go through a serving ring while the
    update worker of Server runs on the update stream.

    slots: ring slots (a query waits for a free slot when all are in use);
    max_us: the lifetime of one ring launch (a launch stops taking queries
    after it, so writer calls, which wait for the last query launch before
    recycling slabs, wait at most that long); blocks: thread blocks of a
    launch (0: one per SM; two launches overlap, leaving room for the update
    kernels).
    """

    def __init__(self, index, k: int = 10, beam: int = 64, slots: int = 4096, max_us: int = 2000,
                 blocks: int = 0, max_update_batch: int = 4096, streams=(None, None), reclaim_every: int = 0,
                 writer_share: float = 0.5):
        super().__init__(index, k=k, beam=beam, max_update_batch=max_update_batch, streams=streams,
                         reclaim_every=reclaim_every)
        self.slots, self.max_us, self.blocks = slots, max_us, blocks
        self.writer_share = writer_share

    def run(self, requests: list[Request]) -> dict:
        """Queries go through the ring (native submit / launch / collect
        threads, etale_ring_serve) while this object's update worker runs on
        the update stream."""
        from .binding import Ring
        queries = [r for r in requests if r.kind == "query"]
        updates = [r for r in requests if r.kind != "query"]
        ring = Ring(self.index, self.slots, self.k, self.beam)
        # one empty launch first: the kernel's first launch in a process also
        # loads it, which would otherwise land on the first arrivals
        import torch
        ring.launch(1, self.blocks, self.qstream)
        torch.cuda.synchronize()
        self.index.set_concurrent(True)
        if hasattr(self.index, "set_writer_share"):
            self.index.set_writer_share(self.writer_share)   # leave the ring room on the SMs
        res = None
        if queries:
            q = np.stack([r.payload for r in queries]).astype(np.float32)
            arr = np.array([r.t for r in queries], dtype=np.float64)
        t0 = time.perf_counter()
        tu = threading.Thread(target=self._update_worker, args=(updates, t0))
        tu.start()
        if queries:
            # the native call counts time from its own start: shift arrivals
            shift = time.perf_counter() - t0
            res = ring.serve(q, np.maximum(arr - shift, 0.0), self.max_us, self.blocks, self.qstream)
            for k, r in enumerate(queries):
                r.issued = res["issued"][k] + shift
                r.done = res["done"][k] + shift
                r.result = (res["ids"][k], res["dists"][k])
        tu.join()
        wall = time.perf_counter() - t0
        self.index.set_concurrent(False)
        if hasattr(self.index, "set_writer_share"):
            self.index.set_writer_share(1.0)
        rs = ring.stats()
        ring.close()
        ql = [r.done - r.t for r in queries]
        ul = [r.done - r.t for r in updates]
        return {"wall_s": wall, "queries": percentiles(ql), "updates": percentiles(ul),
                "query_throughput": len(queries) / wall if wall > 0 else 0.0,
                "update_vectors_per_s": sum(len(r.payload) for r in updates) / wall if wall > 0 else 0.0,
                "ring_launches": res["launches"] if res else 0,
                "queries_taken_mid_launch": res["mid_launch"] if res else 0,
                "ring_seed_ms_per_query": 1e3 * rs["seed_s"] / max(rs["served"], 1),
                "ring_search_ms_per_query": 1e3 * rs["search_s"] / max(rs["served"], 1),
                "update_batches": sum(1 for e in self.log if e[0] == "update"),
                "deferred": self.deferred, "reclaims": self.reclaims}
