"""Work tallies of the writer kernels (etale_get_work): the bytes each
kernel's step of the method must move, counted on the device.  Where the
exact figure follows from the graph before and after a call, it is checked
here: the replacement sets of a delete read N(u) and the members' words for
every deleted u (Algorithm 3), and compaction reads every reference word,
every live list with one tombstone bit per entry, and rewrites each list that
held a tombstone (Sec. 3.3)."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tallies_match_the_graph():
    from paper_2607_02543_gb300 import Index, build
    build.build()
    w = W.scaled(W.SMALL, 3000, n_queries=10, rounds=1)
    plan = W.make_plan(w)
    g = Index(w.dim, w.metric, w.degree, w.capacity + 1000, build_beam=32, mode="deterministic")
    g.insert(plan.base)
    g.reclaim()
    mp = (w.dim + 3) // 4 * 4
    built = g.work(reset=True)
    assert built["prune"][0] > 0 and built["prune"][0] % (4 * mp) == 0   # fp32 candidate rows
    assert built["prune"][1] > 0 and built["offer_fold"][1] > 0
    assert built["refine"][0] % (4 * mp) == 0

    de0, hs0, dg0, _, _ = g.export_graph()
    D = np.arange(5, 3000, 11, dtype=np.uint32)
    assert not de0[D].any()
    g.delete(D)
    after_del = g.work(reset=True)
    deg = dg0[D].astype(np.int64) * hs0[D]
    assert after_del["repair_k"][0] == int(deg.sum()) * 4 * mp
    assert after_del["repair_k"][1] == int((8 + 16 * deg).sum())
    assert after_del["repair_fold"][1] > 0

    de1, hs1, dg1, ids1, _ = g.export_graph()
    nid = g.stats()["next_id"]
    g.reclaim()
    rec = g.work(reset=True)
    de2, hs2, dg2, _, _ = g.export_graph()
    live = (de1 == 0) & (hs1 == 1)
    n1 = dg1.astype(np.int64)
    expect = 8 * nid + int((8 * n1[live] + (n1[live] + 7) // 8).sum())
    R = ids1.shape[1]
    dead = de1.astype(bool)
    for v in np.nonzero(live)[0]:
        lst = ids1[v, :n1[v]]
        if dead[lst].any():
            expect += 8 * int(dg2[v]) + 8
    assert rec["compact"] == (0, expect)
    assert all(v == (0, 0) for k, v in rec.items() if k != "compact")
    assert R == w.degree
