"""Failure detection without faulting the GPU: a bounded device wait that
runs out becomes ETALE_ETIMEOUT and the context stays usable; a pool that
cannot hold an insert is refused before anything changes; the id budget is
enforced (ETALE_ECAPACITY)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2607_02543_gb300 import Index, build, binding
    build.build()
    assert binding.selftest_bounded_wait(1000) == 5          # ETALE_ETIMEOUT
    assert "bounded device wait" in binding.load().etale_last_error(None).decode()
    # the context is still usable: an index builds and answers
    rng = np.random.default_rng(0)
    g = Index(16, "l2", 8, 500, build_beam=16)
    X = rng.normal(size=(300, 16)).astype(np.float32)
    g.insert(X)
    ids, d = g.search(X[:5], 1, 16)
    assert ids[:, 0].tolist() == [0, 1, 2, 3, 4]


def test_small_pool_refused_before_any_change():
    from paper_2607_02543_gb300 import EtaleError, Index
    rng = np.random.default_rng(1)
    g = Index(16, "l2", 8, 1000, build_beam=16, pool_slabs=40, max_batch=10)
    g.insert(rng.normal(size=(4, 16)).astype(np.float32))
    before = g.stats()
    with pytest.raises(EtaleError) as ei:
        g.insert(rng.normal(size=(50, 16)).astype(np.float32))
    assert ei.value.status == 2                                # ETALE_ENOMEM
    after = g.stats()
    assert after["next_id"] == before["next_id"] and after["live"] == before["live"]
    with pytest.raises(EtaleError) as ei:
        Index(16, "l2", 8, 10).insert(rng.normal(size=(11, 16)).astype(np.float32))
    assert ei.value.status == 3                                # ETALE_ECAPACITY
