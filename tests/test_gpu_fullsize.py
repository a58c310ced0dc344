"""Full-size checks at 1,000,000 x 128 (integer-valued mixture, degree 32,
build beam 128, lock-free mode, 1% churn rounds): the oracle cannot hold
this graph, so the CUDA path is checked through properties that hold at any
size and through outputs the oracle and brute force compute one by one."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.graph_checks import NIL, recall_at_k

pytestmark = pytest.mark.gpu

N_ENTRY = 4096
BEAM = 128


@pytest.fixture(scope="module")
def state():
    import torch
    from paper_2607_02543_gb300 import Index, build
    build.build()
    w = W.dataclasses.replace(W.SIFT_LIKE_1M, rounds=2)
    plan = W.make_plan(w)
    dev = torch.device("cuda", 0)
    g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=w.build_beam, mode="lockfree", n_entry=N_ENTRY)
    g.insert(torch.from_numpy(plan.base).to(dev))
    g.reclaim()
    alive = np.zeros(w.capacity, bool)
    alive[:w.n_base] = True
    ever = np.zeros(w.capacity, bool)
    for r in range(w.rounds):
        dele = W.choose_deletes(plan.delete_rng, np.nonzero(alive)[0].astype(np.uint32), w.n_delete)
        assert g.delete(dele) == w.n_delete
        ids = g.insert(torch.from_numpy(plan.inserts[r]).to(dev))
        alive[dele] = False
        alive[ids] = True
        ever[dele] = True
    X = np.concatenate([plan.base] + plan.inserts)
    return g, w, plan, alive, ever, X


def test_invariants_before_reclaim(state, oracle_mod):
    g, w, plan, alive, ever, X = state
    de, hs, dg, ids, rho = g.export_graph()
    n = de.size
    assert (dg <= w.degree).all()
    assert (de.astype(bool) == ever[:n]).all()              # Proposition 1 (flags)
    assert (hs[:n] == 1).all()                              # tombstones keep their slab until reclaim
    rng = np.random.default_rng(5)
    us = rng.choice(np.nonzero(alive[:n])[0], 400, replace=False)
    for u in us:                                            # stored rho is the canonical distance
        for j in range(int(dg[u])):
            a = int(ids[u, j])
            assert a != u and a < n
            assert oracle_mod.dist(X[u], X[a]) == float(rho[u, j])
        k = ids[u, :dg[u]]
        assert np.unique(k).size == k.size


def test_reclaim_footprint_and_search(state, oracle_mod):
    g, w, plan, alive, ever, X = state
    g.reclaim()
    s = g.stats()
    assert s["used_slabs"] == s["live"] == int(alive.sum())  # Proposition 3
    de, hs, dg, ids, rho = g.export_graph()
    live = (de == 0) & (hs == 1)
    mask = np.arange(w.degree)[None, :] < dg[:, None]
    tgt = ids[live][mask[live]]
    assert (de[tgt] == 0).all()                             # no live -> tombstone edge
    q = plan.queries
    got, gd = g.search(q, w.k, BEAM)
    assert not np.isin(got[got != NIL], np.nonzero(ever)[0]).any()
    gt, _ = g.ground_truth(q, w.k)
    rec = recall_at_k(got, gt)
    assert rec >= 0.95, rec
    # sampled outputs computed one by one: returned distances are canonical,
    # and the ground-truth kernel agrees with fp64 brute force
    rng = np.random.default_rng(6)
    live_ids = np.nonzero(alive)[0]
    Xl = X[live_ids].astype(np.float64)
    for t in rng.choice(q.shape[0], 24, replace=False):
        for j in range(w.k):
            if got[t, j] != NIL:
                assert oracle_mod.dist(q[t], X[got[t, j]]) == float(gd[t, j])
        d64 = ((Xl - q[t].astype(np.float64)) ** 2).sum(1)
        top = live_ids[np.argsort(d64, kind="stable")[:w.k]]
        assert set(top.tolist()) == set(gt[t].tolist())
