"""The serving loop on the GPU: continuous batching with a query stream and
an update stream overlapping on the device (concurrent mode)."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.graph_checks import NIL, check_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2607_02543_gb300 import Index, build
    build.build()
    w = W.scaled(W.SMALL, 20000, n_queries=2000, rounds=1)
    plan = W.make_plan(w)
    g = Index(w.dim, w.metric, w.degree, w.capacity + 20000, build_beam=32, mode="lockfree")
    g.insert(plan.base)
    g.reclaim()
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    return g, w, plan, streams


def test_results_same_alone_and_in_the_mix(setup):
    from paper_2607_02543_gb300.serve import Request, Server
    g, w, plan, streams = setup
    alone_ids, alone_d = g.search(plan.queries, 10, 64)
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 0.05, plan.queries.shape[0]))
    reqs = [Request(float(ti), "query", plan.queries[i]) for i, ti in enumerate(t)]
    srv = Server(g, k=10, beam=64, max_query_batch=300, streams=streams)
    srv.run(reqs)
    assert srv.log and max(n for *_, n in srv.log) > 1      # real batches were formed
    for i, r in enumerate(reqs):
        ids, d = r.result
        assert (ids == alone_ids[i]).all() and np.array_equal(d, alone_d[i])


def test_concurrent_updates_keep_invariants(setup, oracle_mod):
    from paper_2607_02543_gb300.serve import Request, Server, overlap_seconds
    g, w, plan, streams = setup
    rng = np.random.default_rng(4)
    dur = 0.6
    reqs = []
    for ti in np.sort(rng.uniform(0, dur, 1500)):
        reqs.append(Request(float(ti), "query", plan.queries[rng.integers(plan.queries.shape[0])]))
    fresh = W.Mixture(w).draw("inserts", 3000)
    live = np.arange(w.n_base, dtype=np.uint32)
    rng.shuffle(live)
    off_i = off_d = 0
    for ti in np.sort(rng.uniform(0, dur, 60)):
        n = int(rng.integers(1, 100))
        if rng.random() < 0.5:
            reqs.append(Request(float(ti), "insert", fresh[off_i:off_i + n]))
            off_i += n
        else:
            reqs.append(Request(float(ti), "delete", live[off_d:off_d + n]))
            off_d += n
    reqs.sort(key=lambda r: r.t)
    srv = Server(g, k=10, beam=64, max_query_batch=512, streams=streams)
    out = srv.run(reqs)
    assert out["queries"]["n"] == 1500 and np.isfinite(out["queries"]["p99_ms"])
    # Proposition 1 under concurrency: a query issued after a delete call
    # returned never sees the deleted ids
    deletes = [r for r in reqs if r.kind == "delete"]
    for r in reqs:
        if r.kind != "query":
            continue
        gone = [d.payload for d in deletes if d.done < r.issued]
        if gone:
            ids = r.result[0]
            assert not np.isin(ids[ids != NIL], np.concatenate(gone)).any()
    g.reclaim()
    check_graph(g.export_graph(), w.degree, after_reclaim=True)
    s = g.stats()
    assert s["used_slabs"] == s["live"]
    print("serving:", out, "overlap_s:", overlap_seconds(srv.log))


def test_ring_results_same_alone_and_in_the_mix(setup):
    """Slot-granular serving: each query's result through the serving ring
    equals etale_search's bit for bit, and some queries are taken by a launch
    that was already running when they arrived."""
    from paper_2607_02543_gb300.serve import Request, RingServer
    g, w, plan, streams = setup
    alone_ids, alone_d = g.search(plan.queries, 10, 64)
    rng = np.random.default_rng(5)
    t = np.sort(rng.uniform(0, 0.08, plan.queries.shape[0]))
    reqs = [Request(float(ti), "query", plan.queries[i]) for i, ti in enumerate(t)]
    srv = RingServer(g, k=10, beam=64, slots=512, max_us=3000, streams=streams)
    out = srv.run(reqs)
    assert out["queries"]["n"] == len(reqs) and out["ring_launches"] >= 2
    assert out["queries_taken_mid_launch"] > 0, out
    for i, r in enumerate(reqs):
        ids, d = r.result
        assert (ids == alone_ids[i]).all() and np.array_equal(d.view(np.uint32), alone_d[i].view(np.uint32)), i


def test_ring_with_concurrent_updates_on_anchor_set(setup):
    """The ring serves an anchor set whose exact neighbours the concurrent
    updates cannot change (deletes avoid those ids; inserts lie far from every
    anchor): recall stays at its quiescent level, no deleted id is returned
    after its delete call returned, and the index keeps its invariants."""
    from paper_2607_02543_gb300.serve import Request, RingServer
    g, w, plan, streams = setup
    anchors = plan.queries[:1000]
    gt, _ = g.ground_truth(anchors, 10)
    protected = np.unique(gt)
    alone, _ = g.search(anchors, 10, 64)
    rec_alone = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(alone.tolist(), gt.tolist())])
    rng = np.random.default_rng(6)
    dur = 0.5
    reqs = [Request(float(ti), "query", anchors[rng.integers(1000)]) for ti in np.sort(rng.uniform(0, dur, 3000))]
    idx_of = {id(r): None for r in reqs}
    de, hs = g.export_graph()[:2]
    live = np.setdiff1d(np.nonzero((de == 0) & (hs == 1))[0], protected).astype(np.uint32)
    rng.shuffle(live)
    fresh = (W.Mixture(w).draw("inserts", 3000) + 1.0e4).astype(np.float32)
    off_i = off_d = 0
    for ti in np.sort(rng.uniform(0, dur, 60)):
        n = int(rng.integers(1, 80))
        if rng.random() < 0.5:
            reqs.append(Request(float(ti), "insert", fresh[off_i:off_i + n]))
            off_i += n
        else:
            reqs.append(Request(float(ti), "delete", live[off_d:off_d + n]))
            off_d += n
    reqs.sort(key=lambda r: r.t)
    srv = RingServer(g, k=10, beam=64, slots=1024, max_us=2000, streams=streams, reclaim_every=4)
    out = srv.run(reqs)
    qs = [r for r in reqs if r.kind == "query"]
    assert out["queries"]["n"] == len(qs) and out["update_batches"] > 0
    row = {a.tobytes(): i for i, a in enumerate(anchors)}
    hits = [len(set(r.result[0].tolist()) & set(gt[row[r.payload.tobytes()]].tolist())) / 10 for r in qs]
    assert np.mean(hits) >= rec_alone - 0.01, (np.mean(hits), rec_alone)
    deletes = [r for r in reqs if r.kind == "delete"]
    for r in qs:
        gone = [d.payload for d in deletes if d.done < r.issued]
        if gone:
            ids = r.result[0]
            assert not np.isin(ids[ids != NIL], np.concatenate(gone)).any()
    g.reclaim()
    check_graph(g.export_graph(), w.degree, after_reclaim=True)
    s = g.stats()
    assert s["used_slabs"] == s["live"]
    print("ring serving:", out)
