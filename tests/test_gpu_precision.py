"""Reduced-precision search copies on the GPU (BF16, per-vector-scaled FP8
E4M3) and the exact fp32 rerank.

The stored codes are integer decisions, so they must equal the reference
codecs (oracle/quant.py) bit for bit.  Reranked results must carry the
canonical fp32 distance exactly.  On integer-valued data of magnitude <= 256
the BF16 copy is lossless, so the BF16 search must equal the fp32 search.
"""
import numpy as np
import pytest

from oracle import quant
from paper_2607_02543_gb300 import workloads as W
from tests.graph_checks import NIL, recall_at_k

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_02543_gb300 import build
    build.build()


def _index(w, plan, **kw):
    from paper_2607_02543_gb300 import Index
    g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=w.build_beam, copies=("bf16", "fp8"), **kw)
    g.insert(plan.base)
    return g


def test_codes_match_reference():
    rng = np.random.default_rng(21)
    from paper_2607_02543_gb300 import Index
    X = rng.normal(0, 3, size=(300, 37)).astype(np.float32)
    X[0] = 0.0                                  # zero row: scale 1
    X[1, 5] = 1e4                               # one large value sets the scale
    X[2] = rng.normal(0, 1e-3, 37)              # tiny values: FP8 subnormals after scaling
    g = Index(37, "l2", 8, 400, build_beam=16, copies=("bf16", "fp8"))
    g.insert(X)
    b, f, sc = g.export_copies(0, 300)
    assert (b == quant.bf16_bits(X)).all()
    for i in range(300):
        codes, s = quant.fp8_row(X[i])
        assert sc[i] == s, i
        assert (f[i] == codes).all(), i


def test_bf16_is_lossless_on_integer_data(oracle_mod):
    w = W.scaled(W.SIFT_LIKE_1M, 3000, n_queries=300)
    plan = W.make_plan(w)
    g = _index(w, plan)
    ids32, d32 = g.search(plan.queries, 10, 64)
    g.set_search_precision("bf16")
    idsb, db = g.search(plan.queries, 10, 64)
    assert (idsb == ids32).all() and np.array_equal(db, d32)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_reranked_search(oracle_mod, prec):
    # unit vectors, inner product (the 768-d text-embedding shape, scaled down)
    w = W.Workload("unit-ip", 4000, 96, "ip", 32, 64, 1, 40, 40, 400, 10, 64, 32, "unit")
    plan = W.make_plan(w)
    g = _index(w, plan)
    gt, _ = g.ground_truth(plan.queries, 10)
    ids32, _ = g.search(plan.queries, 10, 64)
    g.set_search_precision(prec)
    ids, dist = g.search(plan.queries, 10, 64)
    r32, rp = recall_at_k(ids32, gt), recall_at_k(ids, gt)
    assert rp >= r32 - 0.02, (prec, rp, r32)
    # every returned distance is the exact canonical fp32 distance
    for t in range(0, plan.queries.shape[0], 37):
        for j in range(10):
            if ids[t, j] != NIL:
                assert oracle_mod.dist(plan.queries[t], plan.base[ids[t, j]], "ip") == float(dist[t, j])
        row = dist[t][ids[t] != NIL]
        assert (np.diff(row) >= 0).all()
    # a copy that is not kept is refused
    from paper_2607_02543_gb300 import EtaleError, Index
    h = Index(w.dim, w.metric, w.degree, 100)
    with pytest.raises(EtaleError):
        h.set_search_precision(prec)


@pytest.mark.parametrize("dim", [96, 320])
def test_bf16_key_paths(oracle_mod, dim):
    """Both places a BF16 search may take its beam keys from (tensor-core
    dot products, CUDA-core reduction of the widened row) reach the fp32
    search's recall and return exact canonical fp32 distances, in order; the
    autotuner reports which path each shape used."""
    w = W.Workload("unit-ip", 3000, dim, "ip", 32, 64, 1, 40, 40, 300, 10, 64, 32, "unit")
    plan = W.make_plan(w)
    g = _index(w, plan)
    gt, _ = g.ground_truth(plan.queries, 10)
    ids32, _ = g.search(plan.queries, 10, 64)
    r32 = recall_at_k(ids32, gt)
    g.set_search_precision("bf16")
    for tensor in (True, False):
        g.set_search_keys(tensor)
        ids, dist = g.search(plan.queries, 10, 64)
        assert recall_at_k(ids, gt) >= r32 - 0.02, (dim, tensor)
        for t in range(0, plan.queries.shape[0], 29):
            for j in range(10):
                if ids[t, j] != NIL:
                    assert oracle_mod.dist(plan.queries[t], plan.base[ids[t, j]], "ip") == float(dist[t, j])
            row = dist[t][ids[t] != NIL]
            assert (np.diff(row) >= 0).all()
    from paper_2607_02543_gb300 import EtaleError
    with pytest.raises(EtaleError):
        g._check(g.lib.etale_set_search_keys(g.h, 2))
    import torch
    q = torch.from_numpy(plan.queries[:256]).cuda()
    tried = g.autotune_search(q, 10, 64)
    assert {t[4] for t in tried} == {0, 1}
