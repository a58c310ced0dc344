"""The measurements beyond the headline round, on the GPU, checked.

- Proposition 4 / Remark 1 (Sec. 4.5): with tombstones accumulated over churn
  rounds and no Reclaim, the dead-edge and dirty-node counts of the GPU graph
  equal the oracle's on the same inputs (deterministic mode), and Reclaim's
  compaction republishes exactly the dirty nodes (Algorithm 4).
- The reclaim-interval run (f1), the pure-deletion stress (f2, Sec. 5.4) and
  the concurrent-latency run (f3, Sec. 5.5) at a small scale: the properties
  that hold at any size (republications == dirty nodes; used slabs == live
  after every Reclaim, Proposition 3; anchor recall with and without a
  concurrent writer).
"""
import numpy as np
import pytest

from paper_2607_02543_gb300 import experiments as X
from paper_2607_02543_gb300 import workloads as W
from tests.pair import make_pair, graphs_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02543_gb300 import build
    build.build()


def test_dirty_nodes_and_dead_edges_match_oracle(oracle_mod):
    w = W.scaled(W.SMALL, 2000, n_queries=10, rounds=4)
    p = W.make_plan(w)
    g, o = make_pair(oracle_mod, w.dim, w.metric, w.degree, w.capacity, build_beam=32, n_entry=64)
    g.insert(p.base)
    o.insert(p.base)
    rng = np.random.default_rng(11)
    alive = np.zeros(w.capacity, bool)
    alive[:w.n_base] = True
    for r in range(4):        # tombstones accumulate: no Reclaim between rounds
        dele = rng.choice(np.nonzero(alive)[0], 40, replace=False).astype(np.uint32)
        assert g.delete(dele) == o.delete(dele) == 40
        alive[dele] = False
        ids = g.insert(p.inserts[r])
        assert np.array_equal(ids, o.insert(p.inserts[r]))
        alive[ids] = True
        cg, co = X.dead_edge_counts(g.export_graph()), X.dead_edge_counts(o.dump())
        assert cg == co
        assert cg["dead_edges"] > 0 and cg["dirty"] <= cg["dead_edges"]
    pg, po = g.stats()["n_publish"], o.stats()["n_publish"]
    g.reclaim()
    o.reclaim()
    assert not graphs_equal(g.export_graph(), o.dump(), w.degree)
    # Algorithm 4, phase 1: one republication per dirty node, no other
    assert g.stats()["n_publish"] - pg == o.stats()["n_publish"] - po == cg["dirty"]
    after = X.dead_edge_counts(g.export_graph())
    assert after["dead_edges"] == 0
    s = g.stats()
    assert s["used_slabs"] == s["live"]


def test_reclaim_interval_small():
    w = W.scaled(W.SIFT_LIKE_1M, 20_000)
    r = X.run_reclaim_interval(w, rounds=(1, 2, 4, 8))
    pts = r["points"]
    assert [p["rounds"] for p in pts] == [1, 2, 4, 8]
    for a, b in zip(pts, pts[1:]):
        assert b["t"] > a["t"] and b["dead_edges"] > a["dead_edges"]
    for p in pts:
        assert p["republished"] == p["dirty"] <= p["live"]
        assert 0 < p["model_dirty"] <= p["live"]
    assert r["model_tau"] > 0 and r["fit_dead_edges_linear_slope"] > 0


def test_deletion_stress_small():
    w = W.scaled(W.SIFT_LIKE_1M, 20_000, n_queries=200)
    r = X.run_deletion_stress(w, frac=0.2, beam=96)
    rows = r["rounds"]
    assert rows and rows[-1]["live"] <= w.n_base // 2
    for row in rows:
        assert row["used_slabs"] == row["live"]          # Proposition 3 after every Reclaim
        assert row["recall_at_10"] >= 0.9, row


def test_concurrent_latency_small():
    w = W.scaled(W.SIFT_LIKE_1M, 20_000, n_queries=500)
    r = X.run_concurrent_latency(w, batch=200, n_batches=40, beam=96, extra=200_000, n_fresh=100_000)
    assert r["concurrent"]["writer_rounds"] > 0
    for side in ("quiescent", "concurrent"):
        assert r[side]["recall_at_10"] >= 0.9, r
        assert r[side]["p99_ms"] >= r[side]["p50_ms"] > 0
