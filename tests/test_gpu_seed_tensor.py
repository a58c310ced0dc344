"""Entry-set seeding on tensor cores (certified exact rerank) against the
CUDA-core seed kernel: in deterministic mode the two must build bit-identical
graphs and return identical searches, on integer data (exact in bf16) and on
Gaussian and unit-vector data (hi/lo split), at dimensions where the query
tile stays in shared memory and where it streams through the copy ring, with
entry sets smaller and larger than the beam and insert batches above and
below the tensor path's minimum batch."""
import dataclasses

import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests.pair import graphs_equal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wname,n,n_entry,beam", [
    ("int", 6_000, 1024, 64),
    ("gauss", 5_000, 700, 64),
    ("unit", 4_000, 256, 96),
    ("int", 3_000, 40, 64),          # fewer entries than the beam: every entry is a seed
    ("wide", 3_000, 512, 64),        # 300-d: the query tile streams through the ring
    ("gist", 2_000, 300, 48),        # 960-d non-negative mixture, streamed
])
def test_tensor_seeds_build_the_same_graph(wname, n, n_entry, beam):
    from paper_2607_02543_gb300 import Index
    base = {"int": W.SIFT_LIKE_1M, "gauss": W.SMALL,
            "unit": dataclasses.replace(W.SMALL, metric="ip", kind="unit", dim=96),
            "wide": dataclasses.replace(W.SMALL, dim=300), "gist": W.GIST_LIKE_1M}[wname]
    w = dataclasses.replace(W.scaled(base, n, n_queries=500), rounds=2)
    plan = W.make_plan(w)
    out = []
    for seed in ("default", "cuda_cores"):
        g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=beam, n_entry=n_entry, seed=seed)
        g.insert(plan.base)
        for r in range(w.rounds):
            de, hs = g.export_graph()[:2]
            live = np.nonzero((de == 0) & (hs == 1))[0].astype(np.uint32)
            g.delete(live[:: max(1, len(live) // max(1, w.n_delete))][: w.n_delete])
            g.insert(plan.inserts[r][:17])       # below the tensor path's batch minimum
            g.insert(plan.inserts[r][17:])
            g.reclaim()
        ids, d = g.search(plan.queries, 10, beam)
        out.append((g.export_graph(), ids, d))
    (ga, ia, da), (gb, ib, db) = out
    assert graphs_equal(ga, gb, w.degree) == []
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(da.view(np.uint32), db.view(np.uint32))
