"""Recorded churn rounds (etale_round_graph_*).

A round recorded once as a CUDA graph (delete with repair, one insert
sub-batch with refine, Reclaim, a query batch) and replayed with one launch
per round must do exactly what the eager calls do:
- deterministic mode: after every replayed round the graph equals the
  oracle's bit for bit (ids, degrees, flags, rho bits) and the replayed
  queries equal the oracle's search;
- lock-free mode: every invariant, used slabs == live after each round
  (Proposition 3), and Recall@10 >= 0.95;
- eager calls between replays see the right counts; a recorded buffer is
  never reallocated while the graph lives; NIL-padded delete lists work.
"""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.graph_checks import check_graph, recall_at_k, NIL
from tests.pair import make_pair, graphs_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02543_gb300 import build
    build.build()


def _live(dump):
    return np.nonzero((dump[0] == 0) & (dump[1] == 1))[0].astype(np.uint32)


def test_replayed_rounds_equal_oracle(oracle_mod):
    import torch
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SMALL, 3000, n_queries=200, rounds=4)
    p = W.make_plan(w)
    g, o = make_pair(oracle_mod, w.dim, w.metric, w.degree, w.capacity, build_beam=32, n_entry=64)
    g.insert(p.base)
    o.insert(p.base)
    o.reclaim()
    g.reclaim()
    n_del_max = w.n_delete + 7                       # padded with NIL
    d_del = torch.full((n_del_max,), -1, dtype=torch.int32, device=dev)
    d_ins = torch.zeros((w.n_insert, w.dim), dtype=torch.float32, device=dev)
    d_q = torch.from_numpy(p.queries).to(dev)
    out = (torch.empty((w.n_queries, 10), dtype=torch.int32, device=dev),
           torch.empty((w.n_queries, 10), dtype=torch.float32, device=dev))
    rg = g.round_graph(d_del, d_ins, d_q, out, k=10, beam=48)
    for r in range(w.rounds):
        dele = W.choose_deletes(p.delete_rng, _live(o.dump()), w.n_delete)
        pad = np.full(n_del_max, NIL, np.uint32)
        pad[:dele.size] = dele
        if r == 1:
            pad[-1] = dele[0]                          # a repeated id: a no-op
        d_del.copy_(torch.from_numpy(pad.view(np.int32)))
        d_ins.copy_(torch.from_numpy(p.inserts[r]))
        rg.launch()
        o.delete(dele)
        o.insert(p.inserts[r])
        o.reclaim()
        probs = graphs_equal(g.export_graph(), o.dump(), w.degree)   # waits for the replay
        assert not probs, f"round {r}: " + "; ".join(probs)
        assert np.array_equal(g.entries(), o.entries())
        oi, od = o.search(p.queries, 10, 48)
        gi = out[0].cpu().numpy().view(np.uint32)
        gd = out[1].cpu().numpy()
        assert np.array_equal(gi, oi) and np.array_equal(gd.view(np.uint32), od.view(np.uint32))
        s, so = g.stats(), o.stats()
        assert s["live"] == so["live"] and s["used_slabs"] == s["live"] and s["tombstones"] == 0
        assert s["next_id"] == so["next_id"]
    rg.close()


def test_replayed_rounds_lockfree_invariants_and_recall(oracle_mod):
    """Lock-free replays (inserts of 60 rows: tensor-core seeding) keep every
    invariant and stay within 0.005 Recall@10 of the oracle (>= 0.95)."""
    import torch
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SMALL, 6000, n_queries=500, rounds=3)
    p = W.make_plan(w)
    g, _ = make_pair(oracle_mod, w.dim, w.metric, w.degree, w.capacity, build_beam=w.build_beam,
                     mode="lockfree", with_oracle=False)
    o = oracle_mod.Oracle(w.dim, w.metric, w.degree, w.capacity, build_beam=w.build_beam, refine=2)
    g.insert(torch.from_numpy(p.base).to(dev))
    o.insert(p.base)
    g.reclaim()
    o.reclaim()
    d_del = torch.empty((w.n_delete,), dtype=torch.int32, device=dev)
    d_ins = torch.empty((w.n_insert, w.dim), dtype=torch.float32, device=dev)
    d_q = torch.from_numpy(p.queries).to(dev)
    out = (torch.empty((w.n_queries, 10), dtype=torch.int32, device=dev),
           torch.empty((w.n_queries, 10), dtype=torch.float32, device=dev))
    rg = g.round_graph(d_del, d_ins, d_q, out, k=10, beam=64)
    ever = np.zeros(w.capacity, bool)
    for r in range(w.rounds):
        dele = W.choose_deletes(p.delete_rng, _live(o.dump()), w.n_delete)
        d_del.copy_(torch.from_numpy(dele.view(np.int32)))
        d_ins.copy_(torch.from_numpy(p.inserts[r]))
        rg.launch()
        assert o.delete(dele) == dele.size
        o.insert(p.inserts[r])
        o.reclaim()
        ever[dele] = True
    rg.sync()
    dump = g.export_graph()
    n = dump[0].shape[0]
    assert n == o.stats()["next_id"]
    check_graph(dump, w.degree, after_reclaim=True)
    assert (dump[0][ever[:n]] == 1).all() and np.array_equal(_live(dump), _live(o.dump()))
    s = g.stats()
    assert s["used_slabs"] == s["live"] == o.stats()["live"]
    ids = out[0].cpu().numpy().view(np.uint32)
    assert not np.isin(ids[ids != NIL], np.nonzero(ever)[0]).any()
    gt, _ = o.exact_knn(p.queries, 10)
    oi, _ = o.search(p.queries, 10, 64)
    rg_, ro = recall_at_k(ids, gt), recall_at_k(oi, gt)
    assert rg_ >= 0.95 and abs(rg_ - ro) <= 0.005, (rg_, ro)
    rg.close()


def test_eager_calls_between_replays_and_pinned_scratch():
    import torch
    from paper_2607_02543_gb300 import EtaleError, Index
    dev = torch.device("cuda", 0)
    w = W.scaled(W.SMALL, 4000, n_queries=50, rounds=4)
    p = W.make_plan(w)
    g = Index(w.dim, w.metric, w.degree, w.capacity + 2000, build_beam=32, n_entry=64, mode="lockfree")
    g.insert(p.base)
    d_del = torch.arange(100, 120, dtype=torch.int32, device=dev)
    d_ins = torch.from_numpy(p.inserts[0][:20].copy()).to(dev)
    rg = g.round_graph(d_del, d_ins)
    rg.launch()
    # an eager delete waits for the replay and sees its effects
    assert g.delete(np.arange(110, 130, dtype=np.uint32)) == 10     # 110..119 already gone
    s = g.stats()
    assert s["next_id"] == w.n_base + 20 and s["tombstones"] == 10
    # an eager delete larger than the recorded one needs bigger scratch: refused
    with pytest.raises(EtaleError, match="ENOMEM"):
        g.delete(np.arange(1000, 1030, dtype=np.uint32))
    d_del.copy_(torch.arange(200, 220, dtype=torch.int32))
    d_ins.copy_(torch.from_numpy(p.inserts[1][:20]))
    rg.launch()
    rg.sync()
    s = g.stats()
    assert s["tombstones"] == 0 and s["used_slabs"] == s["live"] == w.n_base + 40 - 50
    assert s["next_id"] == w.n_base + 40
    assert g.lib.etale_destroy(g.h) == 1                              # graphs first
    rg.close()
    assert g.delete(np.arange(1000, 1030, dtype=np.uint32)) == 30    # unpinned now
    g.reclaim()
    s = g.stats()
    assert s["used_slabs"] == s["live"] == w.n_base + 40 - 80
