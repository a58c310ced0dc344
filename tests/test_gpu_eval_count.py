"""The search's evaluation count against the oracle's exact visited set.

The BeamSearch kernel keeps a lossy cache of evaluated ids, so it may compute
a distance twice; the method (Sec. 3.4.1, a visited set) computes each once.
etale_search_eval_count logs every evaluation and counts the distinct ids per
query, seeds excluded.  In deterministic mode, with an entry set no larger
than the beam, that count must equal the oracle's distance count for the same
searches minus |E| per query, and the expansions must be equal, whatever the
cache size.  The bench's algorithmic bytes use this count.
"""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.pair import make_pair, churn_round

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02543_gb300 import build
    build.build()


@pytest.mark.parametrize("n_entry,beam,seen_bits", [(32, 48, 8), (64, 64, 6), (16, 96, 10)])
def test_unique_evaluations_equal_oracle_distance_count(oracle_mod, n_entry, beam, seen_bits):
    w = W.scaled(W.SMALL, 3000, n_queries=300, rounds=1)
    p = W.make_plan(w)
    g, o = make_pair(oracle_mod, w.dim, w.metric, w.degree, w.capacity, build_beam=32, n_entry=n_entry)
    g.insert(p.base)
    o.insert(p.base)
    churn_round(g, o, p, 0, w.n_delete, reclaim=False)   # tombstones relay in the searches
    g.set_search_tuning(8, seen_bits)
    s0 = o.stats()
    oi, od = o.search(p.queries, 10, beam)
    s1 = o.stats()
    gi, gd = g.search(p.queries, 10, beam)
    assert np.array_equal(gi, oi) and np.array_equal(gd.view(np.uint32), od.view(np.uint32))
    c = g.eval_count(p.queries, 10, beam)
    S = len(o.entries())
    assert S <= beam
    nq = p.queries.shape[0]
    assert c["n_expand"] == s1["n_expand"] - s0["n_expand"]
    assert c["n_unique"] == s1["n_dist"] - s0["n_dist"] - nq * S
    assert c["n_eval"] >= c["n_unique"]
