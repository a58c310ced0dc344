"""Host-side pieces of the measurements (no GPU): Proposition 4's uniform
model against its own Monte-Carlo and its closed limits, the saturating fit
on known parameters, and the dead-edge count on a hand-made graph."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import experiments as X


def test_dirty_model_limits_and_monte_carlo():
    L, dbar = 10_000, 32.0
    assert X.dirty_model(L, dbar, 0) == 0.0
    assert X.dirty_model(L, dbar, 10 * L) == pytest.approx(L, rel=1e-6)
    # small t: each stranded edge lands on a fresh node, D ~ dbar * t
    assert X.dirty_model(L, dbar, 1) == pytest.approx(dbar, rel=0.01)
    rng = np.random.default_rng(0)
    for t in (10, 100, 500):
        draws = [X.dirty_monte_carlo(L, dbar, t, rng) for _ in range(200)]
        mean, sd = np.mean(draws), np.std(draws) / np.sqrt(len(draws))
        assert abs(mean - X.dirty_model(L, dbar, t)) < 4 * sd + 1e-9, (t, mean)


def test_fit_saturating_recovers_parameters():
    t = np.array([1e3, 2e3, 5e3, 1e4, 2e4, 5e4, 1e5, 2e5])
    y = 37.0 * (1.0 - np.exp(-t / 3.1e4))
    f = X.fit_saturating(t, y)
    assert f["M"] == pytest.approx(37.0, rel=1e-4)
    assert f["tau"] == pytest.approx(3.1e4, rel=1e-4)
    assert f["r2"] > 0.999999


def test_dead_edge_counts_hand_graph():
    # nodes 0..4; 3 is a tombstone (deleted, slab kept), 4 reclaimed (deleted, no slab)
    deleted = np.array([0, 0, 0, 1, 1], np.uint8)
    has_slab = np.array([1, 1, 1, 1, 0], np.uint8)
    degree = np.array([2, 2, 1, 1, 0], np.uint8)
    ids = np.array([[1, 3], [3, 2], [0, 0], [0, 0], [0, 0]], np.uint32)
    rho = np.zeros((5, 2), np.float32)
    c = X.dead_edge_counts((deleted, has_slab, degree, ids, rho))
    assert c == {"live": 3, "live_edges": 5, "dead_edges": 2, "dirty": 2}
