"""Ground truth on tensor cores (tcgen05 candidate pass + certified exact
rerank) against the CUDA-core exact kernel (bit-exact ids and distance
bits) and against the oracle's brute force, on the three mixture families:
integer data (exact in bf16: one bf16 segment), Gaussian data (hi/lo split)
and unit vectors under inner product.  Sizes span several 128-row tiles with
a ragged tail, a ragged query tile, and deleted rows."""
import dataclasses

import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair_indices(w, n, deleted_every, **kw):
    from paper_2607_02543_gb300 import Index
    plan = W.make_plan(dataclasses.replace(W.scaled(w, n, n_queries=333), rounds=0))
    out = []
    for gt in ("default", "cuda_cores"):
        g = Index(w.dim, w.metric, w.degree, n + 10, build_beam=16, max_cand=32, gt=gt, **kw)
        g.insert(plan.base)
        if deleted_every:
            g.delete(np.arange(0, n, deleted_every, dtype=np.uint32))
        out.append(g)
    return plan, out


@pytest.mark.parametrize("wname,n,k,path", [
    ("int", 5_000 + 77, 10, "tensor"),
    ("gauss", 4_000 + 5, 10, "tensor_split"),
    ("unit", 3_000 + 31, 7, "tensor_split"),
    ("int", 300, 32, "tensor"),
    ("wide", 2_000 + 3, 10, "tensor_split"),    # 300-d: the query tile streams through the ring
    ("gist", 1_500 + 11, 10, "tensor_split"),   # 960-d non-negative mixture, streamed
])
def test_tensor_ground_truth_matches_exact(oracle_mod, wname, n, k, path):
    base = {"int": W.SIFT_LIKE_1M, "gauss": W.SMALL,
            "unit": dataclasses.replace(W.SMALL, metric="ip", kind="unit", dim=96),
            "wide": dataclasses.replace(W.SMALL, dim=300), "gist": W.GIST_LIKE_1M}[wname]
    plan, (gt_tc, gt_cc) = _pair_indices(base, n, 9)
    ti, td = gt_tc.ground_truth(plan.queries, k)
    info = gt_tc.ground_truth_info()
    ci, cd = gt_cc.ground_truth(plan.queries, k)
    assert gt_cc.ground_truth_info()["path"] == "cuda_cores"
    assert info["path"] == path
    np.testing.assert_array_equal(ti, ci)
    np.testing.assert_array_equal(td.view(np.uint32), cd.view(np.uint32))
    if k <= 16:   # with k = 32 = the candidate count there is no margin to certify
        assert info["fallback_queries"] <= len(plan.queries) // 10, info
    # the oracle ranks in fp64: equal ids up to fp32 ties, close distances
    o = oracle_mod.Oracle(base.dim, base.metric, base.degree, n + 10, build_beam=16)
    o.insert(plan.base)
    o.delete(np.arange(0, n, 9, dtype=np.uint32))
    oi, od = o.exact_knn(plan.queries, k)
    assert (ti == oi).mean() > 0.999
    assert np.allclose(td, od, rtol=1e-5, atol=1e-5)


def test_tensor_ground_truth_few_live_rows():
    """Fewer live rows than k: padded with NIL / +inf like the exact kernel."""
    from paper_2607_02543_gb300 import Index, NIL
    rng = np.random.default_rng(3)
    X = rng.integers(0, 255, size=(20, 128)).astype(np.float32)
    g = Index(128, "l2", 8, 100, build_beam=16)
    g.insert(X)
    g.delete(np.arange(0, 20, 2, dtype=np.uint32))
    ids, d = g.ground_truth(X[:50], 16)
    assert g.ground_truth_info()["path"] == "tensor"
    assert (ids[:, 10:] == NIL).all() and np.isinf(d[:, 10:]).all()
    assert set(ids[0, :10].tolist()) == set(range(1, 20, 2))
