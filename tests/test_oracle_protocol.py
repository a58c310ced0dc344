"""Pins of the oracle's update protocols (Algorithms 1-4) on CPU.

1. A five-point example whose every step is derived by hand below (the
   expected values live in tests/golden/line5_hand.json).
2. Brute force: a search whose beam covers the live set returns the exact k
   nearest live nodes (fp64), before and after deletions.
3. The paper's invariants under seeded churn: deletion monotonicity
   (Proposition 1), degree bound, no live -> tombstone edge after Reclaim,
   footprint == live after Reclaim (Proposition 3), pool conservation.
"""
import json
import os

import numpy as np
import pytest

from tests.graph_checks import check_graph, reachable_from, recall_at_k, NIL
from paper_2607_02543_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "line5_hand.json")

# ---------------------------------------------------------------------------
# Hand derivation (R = 2, alpha = 1, E = {smallest live id}, one node per
# sub-batch, no refine).  Points x = 0, 10, 1, 11, 5 on the first axis;
# squared distances are exact integers.
#
# id0 (x=0):  empty graph -> F = {} -> publish [].
# id1 (x=10): E = {0}; beam [0(100)]; expand 0: no neighbours.  C = {0}.
#             F = [0(100)].  Offer 1 -> 0: N(0) = [] below R -> [1(100)].
# id2 (x=1):  beam [0(1)]; expand 0 -> 1: d(1,10)=81 -> [0(1), 1(81)];
#             expand 1 -> 0 visited.  C = {0(1), 1(81)}.  Prune: keep 0;
#             1: d(0,1)... d(x0,x1)=100 <= 81? no -> keep.  F = [0(1), 1(81)].
#             Offers: 0 gets 2: [1(100)] -> [2(1), 1(100)];
#                     1 gets 2: [0(100)] -> [2(81), 0(100)].
# id3 (x=11): beam [0(121)]; expand 0 -> 2: d=100, 1: d=1 ->
#             [1(1), 2(100), 0(121)]; expand 1 (2, 0 visited); expand 2.
#             C = 1(1), 2(100), 0(121).  Prune: keep 1; 2: d(10,1)=81 <= 100
#             -> dropped; 0: d(10,0)=100 <= 121 -> dropped.  F = [1(1)].
#             Offer 1 <- 3: N(1) = [2(81), 0(100)] is full -> prune
#             {3(1), 2(81), 0(100)} about x=10: keep 3; 2: d(11,1)=100 <= 81?
#             no; 0: d(11,0)=121 <= 100? no; keep 2 -> R reached: [3(1), 2(81)].
# id4 (x=5):  beam [0(25)]; expand 0 -> 2: d=16, 1: d=25 -> [2(16), 0(25),
#             1(25)] (tie 25 broken by id); expand 2 (0, 1 visited);
#             expand 1 -> 3: d=36 -> [2(16), 0(25), 1(25), 3(36)]; expand 3.
#             C = 2(16), 0(25), 1(25), 3(36).  Prune: keep 2; 0: d(1,0)=1 <=
#             25 -> dropped; 1: d(1,10)=81 <= 25? no; 3: d(1,11)=100 <= 36? no;
#             keep 1 -> R reached.  F = [2(16), 1(25)].
#             Offer 1 <- 4: [3(1), 2(81)] full -> prune {3(1), 4(25), 2(81)}
#             about x=10: keep 3; 4: d(11,5)=36 <= 25? no; 2: 100 <= 81? no;
#             keep 4 -> [3(1), 4(25)].
#             Offer 2 <- 4: [0(1), 1(81)] full -> prune {0(1), 4(16), 1(81)}
#             about x=1: keep 0; 4: d(0,5)=25 <= 16? no; 1: 100 <= 81? no;
#             keep 4 -> [0(1), 4(16)].
# Delete 2:   tombstone 2.  B = N(2) = [0, 4].
#             a=0: K = prune_0({4}) = [4(25)]; N = prune_0(([2(1), 1(100)] \ {2})
#             u K) = prune_0({4(25), 1(100)}): keep 4; 1: d(5,10)=25 <= 100 ->
#             dropped.  -> [4(25)].
#             a=4: K = prune_4({0}) = [0(25)]; N = prune_4({1(25)} u {0(25)}):
#             order 0(25), 1(25); keep 0; 1: d(0,10)=100 <= 25? no -> [0(25), 1(25)].
# Reclaim:    E = {0}; no live list names 2 -> no compaction; 2 -> <1,0,NIL>.
#             used slabs = live = 4.
# Query x=6, k=2, beam 8: from 0 (36): expand 0 -> 4: d=1; expand 4 -> 1: d=16;
#             expand 1 -> 3: d=25; expand 3; expand 0.  Result [4(1), 1(16)].
# ---------------------------------------------------------------------------


def _check_lists(o, expect):
    for u, (ids, rho) in expect.items():
        de, hs, got_ids, got_rho = o.node(int(u))
        assert hs
        assert got_ids.tolist() == ids, (u, got_ids, ids)
        assert got_rho.tolist() == [float(r) for r in rho], (u, got_rho, rho)


def test_hand_derived_line(oracle_mod):
    g = json.load(open(GOLD))
    X = np.zeros((5, g["dim"]), np.float32)
    X[:, 0] = g["points_x"]
    o = oracle_mod.Oracle(g["dim"], "l2", g["degree"], 100, build_beam=g["build_beam"],
                          alpha=g["alpha"], refine=g["refine"], max_batch=g["max_batch"],
                          n_entry=g["n_entry"])
    ids = o.insert(X)
    assert ids.tolist() == [0, 1, 2, 3, 4]
    _check_lists(o, g["after_inserts"])
    assert o.delete(g["delete"]) == 1
    _check_lists(o, g["after_delete"])
    assert [o.node(u)[0] for u in range(5)] == g["deleted_flags_after_delete"]
    o.reclaim()
    s = o.stats()
    assert s["live"] == g["after_reclaim_live"]
    assert s["used_slabs"] == g["after_reclaim_used_slabs"]
    assert s["tombstones"] == 0 and s["reclaimed"] == 1
    q = np.zeros((1, g["dim"]), np.float32)
    q[0, 0] = g["query_x"]
    rid, rd = o.search(q, g["k"], g["beam"])
    assert rid[0].tolist() == g["query_result"][0]
    assert rd[0].tolist() == [float(x) for x in g["query_result"][1]]


def _small_index(oracle_mod, n, refine=2, seed_shift=0, **kw):
    w = W.scaled(W.SMALL, n, n_queries=200)
    p = W.make_plan(w)
    o = oracle_mod.Oracle(w.dim, "l2", w.degree, w.capacity, build_beam=w.build_beam,
                          refine=refine, **kw)
    o.insert(p.base)
    o.reclaim()
    return w, p, o


def test_full_beam_search_is_exact_knn(oracle_mod):
    # With the beam as large as the live set and every live node reachable,
    # BeamSearch evaluates every live node, so the top-k equals brute force.
    w, p, o = _small_index(oracle_mod, 300, n_entry=8)
    dump = o.dump()
    assert reachable_from(dump, o.entries())[dump[0] == 0].all()
    X = p.base
    for phase in range(2):
        q = p.queries[:50]
        ids, d = o.search(q, 10, 400)
        live = np.nonzero(dump[0] == 0)[0]
        D = ((q[:, None, :].astype(np.float64) - X[None, live].astype(np.float64)) ** 2).sum(-1)
        order = np.argsort(D, axis=1, kind="stable")[:, :10]
        assert (ids == live[order]).all()
        ref = np.take_along_axis(D, order, 1)
        assert np.allclose(d, ref, rtol=1e-5, atol=0)
        # delete a third of the live set; tombstones relay, results stay exact
        dele = live[::3].astype(np.uint32)
        o.delete(dele)
        dump = o.dump()
        assert reachable_from(dump, o.entries())[dump[0] == 0].all()
        ids2, _ = o.search(q, 10, 400)
        assert not np.isin(ids2, dele).any()


@pytest.mark.parametrize("refine", [0, 2])
def test_invariants_under_churn(oracle_mod, refine):
    w, p, o = _small_index(oracle_mod, 1500, refine=refine)
    X = np.concatenate([p.base] + p.inserts)
    R = w.degree
    check_graph(o.dump(), R, after_reclaim=True, vectors=X, dist=oracle_mod.dist,
                sample=200)
    ever_deleted = np.zeros(w.capacity, bool)
    next_expected = w.n_base
    for r in range(3):
        de = o.dump()[0]
        live = np.nonzero(de == 0)[0].astype(np.uint32)
        dele = W.choose_deletes(p.delete_rng, live, w.n_delete)
        assert o.delete(dele) == dele.size
        assert o.delete(dele) == 0          # repeat is a no-op
        ever_deleted[dele] = True
        ids = o.insert(p.inserts[r])
        assert ids.tolist() == list(range(next_expected, next_expected + w.n_insert))
        next_expected += w.n_insert
        d1 = o.dump()
        check_graph(d1, R, vectors=X, dist=oracle_mod.dist, sample=100)
        n = d1[0].shape[0]
        # Proposition 1: a deleted id keeps delta = 1 and is never returned
        assert (d1[0][ever_deleted[:n]] == 1).all()
        qi, _ = o.search(p.queries, 10, 64)
        assert not np.isin(qi[qi != NIL], np.nonzero(ever_deleted)[0]).any()
        o.reclaim()
        d2 = o.dump()
        info = check_graph(d2, R, after_reclaim=True)
        s = o.stats()
        # Proposition 3: right after Reclaim the resident slab count is L
        assert s["used_slabs"] == s["live"] == info["live"]
        assert s["free_slabs"] + s["retired_slabs"] + s["used_slabs"] == s["pool"]
        assert (d2[0][ever_deleted[:n]] == 1).all()
        assert reachable_from(d2, o.entries())[d2[0] == 0].mean() > 0.99


def test_recall_small_scale(oracle_mod):
    # The paper reports Recall@10 in 0.95-0.99 at 1% churn (Sec. 5.3); the
    # oracle on a 2,000-point slice of the 64-cluster mixture must reach it.
    w, p, o = _small_index(oracle_mod, 2000, refine=2)
    gt, _ = o.exact_knn(p.queries, 10)
    got, _ = o.search(p.queries, 10, 64)
    assert recall_at_k(got, gt) >= 0.95


def test_capacity_and_empty(oracle_mod):
    o = oracle_mod.Oracle(8, "l2", 4, 10, build_beam=8, refine=0)
    ids, d = o.search(np.zeros((2, 8), np.float32), 3, 8)
    assert (ids == NIL).all() and np.isinf(d).all()
    o.insert(np.random.default_rng(0).normal(size=(10, 8)))
    with pytest.raises(RuntimeError):
        o.insert(np.zeros((1, 8), np.float32))
    assert o.delete([3, 3, 3, 99999]) == 1   # repeats and unknown ids are no-ops
    o.delete(np.arange(10, dtype=np.uint32))
    o.reclaim()
    s = o.stats()
    assert s["live"] == 0 and s["used_slabs"] == 0 and s["n_entries"] == 0
    ids, _ = o.search(np.zeros((1, 8), np.float32), 3, 8)
    assert (ids == NIL).all()
