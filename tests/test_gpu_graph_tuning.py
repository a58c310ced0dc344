"""Launch-shape tuning and CUDA-graph query batches (persistent-round row of
the hot path): results must not depend on the launch shape, and one captured
graph must answer every batch size exactly as etale_search does, also after
the index has been updated."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index():
    import torch
    from paper_2607_02543_gb300 import Index, build
    build.build()
    w = W.scaled(W.SMALL, 6000, n_queries=1000, rounds=1)
    plan = W.make_plan(w)
    g = Index(w.dim, w.metric, w.degree, w.capacity + 1000, build_beam=48, mode="lockfree")
    g.insert(plan.base)
    g.reclaim()
    return g, w, plan, torch.device("cuda", 0)


def test_launch_shapes_do_not_change_results(index):
    import torch
    g, w, plan, dev = index
    q = torch.from_numpy(plan.queries).to(dev)
    ref = g.search(q, 10, 64)
    for rows, bits, wpb in [(8, 8, 4), (16, 9, 2), (32, 11, 8), (4, 12, 2), (8, 8, 8)]:
        g.set_search_tuning(rows, bits, wpb)
        ids, d = g.search(q, 10, 64)
        assert torch.equal(ids, ref[0]) and torch.equal(d, ref[1]), (rows, bits, wpb)
    tried = g.autotune_search(q, 10, 64)
    assert len(tried) >= 6 and all(t[2] > 0 for t in tried)
    assert {t[3] for t in tried} == {2, 4, 8}
    ids, d = g.search(q, 10, 64)
    assert torch.equal(ids, ref[0]) and torch.equal(d, ref[1])


def test_one_graph_serves_every_batch_size(index):
    import torch
    g, w, plan, dev = index
    nq_max, k, beam = 512, 10, 64
    qbuf = torch.zeros((nq_max, w.dim), dtype=torch.float32, device=dev)
    oid = torch.empty((nq_max, k), dtype=torch.int32, device=dev)
    od = torch.empty((nq_max, k), dtype=torch.float32, device=dev)
    nq = torch.zeros(1, dtype=torch.int32, device=dev)
    graph = g.search_graph(qbuf, oid, od, nq, k, beam)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(9)
    for rnd in range(2):
        for n in (1, 7, 300, 512):
            sel = rng.choice(plan.queries.shape[0], n, replace=False)
            qbuf[:n] = torch.from_numpy(plan.queries[sel]).to(dev)
            nq.fill_(n)
            torch.cuda.synchronize()
            graph.launch(stream)
            graph.check(stream)
            ref_ids, ref_d = g.search(plan.queries[sel], k, beam)
            assert (oid[:n].cpu().numpy().view(np.uint32) == ref_ids).all()
            assert np.array_equal(od[:n].cpu().numpy(), ref_d)
        # update the index (the entry set changes); the same graph follows
        g.delete(np.arange(0, 6000, 5, dtype=np.uint32))
        g.insert(W.Mixture(w).draw("inserts", 300))
        g.reclaim()
    graph.close()


def test_autotune_beam_picks_smallest_beam_for_target(index):
    import torch
    g, w, plan, dev = index
    q = torch.from_numpy(plan.queries).to(dev)
    beams = (16, 24, 32, 48, 64, 96)
    chosen, tried = g.autotune_beam(q, 10, 0.97, beams)
    gt, _ = g.ground_truth(q, 10)
    gt = gt.cpu().numpy().view(np.uint32)

    def recall(b):
        ids, _ = g.search(q, 10, b)
        got = ids.cpu().numpy().view(np.uint32)
        return float(np.mean([len(set(a.tolist()) & set(c.tolist())) / 10 for a, c in zip(got, gt)]))

    assert [b for b, _ in tried] == list(beams[:len(tried)])
    for b, r in tried:
        assert abs(r - recall(b)) < 1e-6, (b, r)
    if tried[-1][1] >= 0.97:
        assert chosen == tried[-1][0] and all(r < 0.97 for _, r in tried[:-1])
    else:
        assert chosen == beams[-1] and len(tried) == len(beams)


def test_writer_share_does_not_change_results():
    """Update kernels sized for a share of the SMs build the same graph, word
    for word, in deterministic mode."""
    from paper_2607_02543_gb300 import Index
    w = W.scaled(W.SMALL, 4000, n_queries=10, rounds=1)
    plan = W.make_plan(w)
    out = []
    for share in (1.0, 0.2):
        g = Index(w.dim, w.metric, w.degree, w.capacity + 1000, build_beam=32, mode="deterministic")
        g.set_writer_share(share)
        g.insert(plan.base)
        g.delete(np.arange(0, 4000, 7, dtype=np.uint32))
        g.insert(W.Mixture(w).draw("inserts", 500))
        g.reclaim()
        out.append(g.export_graph())
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_graph_with_tensor_seeds_at_960_dims():
    """A query graph on a 960-d index seeds on tensor cores (the query tile
    streamed through the copy ring, the batch size read on the device) and
    returns what etale_search returns for every batch size."""
    import torch
    from paper_2607_02543_gb300 import Index
    w = W.scaled(W.GIST_LIKE_1M, 2000, n_queries=256, rounds=1)
    plan = W.make_plan(w)
    dev = torch.device("cuda", 0)
    g = Index(w.dim, w.metric, w.degree, w.capacity, build_beam=32, n_entry=256, mode="deterministic")
    g.insert(plan.base)
    nq_max, k, beam = 256, 10, 48
    qbuf = torch.zeros((nq_max, w.dim), dtype=torch.float32, device=dev)
    oid = torch.empty((nq_max, k), dtype=torch.int32, device=dev)
    od = torch.empty((nq_max, k), dtype=torch.float32, device=dev)
    nq = torch.zeros(1, dtype=torch.int32, device=dev)
    graph = g.search_graph(qbuf, oid, od, nq, k, beam)
    stream = torch.cuda.Stream()
    for n in (1, 40, 129, 256):
        qbuf[:n] = torch.from_numpy(plan.queries[:n]).to(dev)
        nq.fill_(n)
        torch.cuda.synchronize()
        graph.launch(stream)
        graph.check(stream)
        ref_ids, ref_d = g.search(plan.queries[:n], k, beam)
        assert (oid[:n].cpu().numpy().view(np.uint32) == ref_ids).all(), n
        assert np.array_equal(od[:n].cpu().numpy().view(np.uint32), ref_d.view(np.uint32)), n
    graph.close()
    g.close()
