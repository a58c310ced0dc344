"""Host checks of the seeded workload generators shared by both sides."""
import numpy as np

from paper_2607_02543_gb300 import workloads as W


def test_absgauss_mixture_is_nonnegative_and_seeded():
    w = W.dataclasses.replace(W.GIST_LIKE_1M, n_base=200, n_clusters=8)
    a = W.Mixture(w).draw("base", 200)
    b = W.Mixture(w).draw("base", 200)
    assert a.shape == (200, 960) and a.dtype == np.float32
    assert (a >= 0).all()
    assert np.array_equal(a, b)
    # centres are |N(0, 10^2)|: the mean coordinate sits near 10 * sqrt(2 / pi) ~ 8
    assert 6.0 < float(a.mean()) < 10.0


def test_uneven_batch_sizes_stay_in_range():
    rng = W._streams(W.GIST_LIKE_1M.seed)["batches"]
    ins = W.random_batch_sizes(rng, 1000, 64, 65_536)
    q = W.random_batch_sizes(rng, 1000, 1, 16_384)
    assert ins.min() >= 64 and ins.max() <= 65_536
    assert q.min() >= 1 and q.max() <= 16_384
    # log-uniform: about half the draws fall below the geometric midpoint
    assert 0.4 < float(np.mean(ins < np.sqrt(64 * 65_536))) < 0.6


def test_appending_a_stream_keeps_earlier_streams():
    w = W.SMALL
    s = W._streams(w.seed)
    import numpy.random as npr
    ss = npr.SeedSequence(w.seed)
    first = npr.Generator(npr.PCG64(ss.spawn(1)[0]))
    assert np.array_equal(s["centers"].normal(size=4), first.normal(size=4))
