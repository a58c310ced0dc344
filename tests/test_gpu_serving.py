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
