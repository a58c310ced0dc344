"""Inserts whose BeamSearch runs on the BF16 or FP8 copies (Algorithm 2 with
reduced-precision search distances; the candidates are re-scored in fp32
before RobustPrune).

- Integer-valued rows of magnitude <= 256 are exact in BF16, so BF16
  searches compute the canonical distances bit for bit: the graph must equal
  the oracle's (fp32) bit for bit, through churn rounds, in deterministic
  mode.  This exercises the re-scoring step with a known answer.
- On Gaussian data the candidate sets change, but every stored rho must be
  the canonical fp32 distance, every invariant must hold, and Recall@10 must
  stay within 0.02 of an index built with fp32 searches.
"""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.graph_checks import check_graph, recall_at_k
from tests.pair import make_pair, graphs_equal, churn_round

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02543_gb300 import build
    build.build()


def test_bf16_inserts_equal_oracle_on_integer_data(oracle_mod):
    from paper_2607_02543_gb300 import Index
    w = W.scaled(W.SIFT_LIKE_1M, 1500, n_queries=100, rounds=2)
    p = W.make_plan(w)
    o = oracle_mod.Oracle(w.dim, w.metric, w.degree, w.capacity, build_beam=64, refine=2, n_entry=128)
    g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=64, n_entry=128, copies=("bf16",))
    g.set_insert_precision("bf16")
    g.insert(p.base)
    o.insert(p.base)
    assert not graphs_equal(g.export_graph(), o.dump(), w.degree)
    for r in range(w.rounds):
        churn_round(g, o, p, r, w.n_delete)
        probs = graphs_equal(g.export_graph(), o.dump(), w.degree)
        assert not probs, f"round {r}: " + "; ".join(probs)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_reduced_precision_inserts_keep_exact_rho_and_recall(oracle_mod, prec):
    from paper_2607_02543_gb300 import Index
    w = W.scaled(W.SMALL, 3000, n_queries=300, rounds=2)
    p = W.make_plan(w)
    X = np.concatenate([p.base] + p.inserts)
    recalls = {}
    for form in ("fp32", prec):
        g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=64, mode="lockfree", copies=("bf16", "fp8"))
        g.set_insert_precision(form)
        g.insert(p.base)
        rng = np.random.default_rng(3)
        for r in range(w.rounds):
            g.delete(rng.choice(w.n_base, w.n_delete, replace=False).astype(np.uint32))
            g.insert(p.inserts[r])
            g.reclaim()
        dump = g.export_graph()
        check_graph(dump, w.degree, after_reclaim=True, vectors=X, dist=oracle_mod.dist, sample=300)
        s = g.stats()
        assert s["used_slabs"] == s["live"]
        gt, _ = g.ground_truth(p.queries, 10)
        ids, _ = g.search(p.queries, 10, 64)
        recalls[form] = recall_at_k(ids, gt)
    assert recalls[prec] >= recalls["fp32"] - 0.02, recalls
