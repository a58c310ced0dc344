"""Pins of the oracle's RobustPrune (Sec. 3.4.1, the slack-alpha rule of DiskANN).

Checked against hand-derived cases, against a library sort when nothing can
dominate (alpha -> infinity), and against the rule's defining certificate in
exact integer arithmetic.
"""
import itertools
import math

import numpy as np
import pytest


def _pad(pts, m=4):
    a = np.zeros((len(pts), m), np.float32)
    for i, p in enumerate(pts):
        a[i, :len(p)] = p
    return a


def test_hand_case_two_dimensions(oracle_mod):
    # Owner at the origin; candidates (1,0), (2,0), (0,1.5), alpha = 1.
    # Squared distances to the owner: 1, 4, 2.25.  Sorted: id0 (1), id2 (2.25), id1 (4).
    # Head id0 is kept.  id2: d(id0, id2) = 1 + 2.25 = 3.25 > 2.25 -> survives.
    # id1: d(id0, id1) = 1 <= 4 -> dominated.  Next head id2 is kept.
    owner = _pad([(0, 0)])[0]
    cand = _pad([(1, 0), (2, 0), (0, 1.5)])
    ids, rho = oracle_mod.robust_prune_vectors(owner, cand, [0, 1, 2], R=8, alpha=1.0)
    assert ids.tolist() == [0, 2]
    assert rho.tolist() == [1.0, 2.25]


def test_hand_case_alpha_slack(oracle_mod):
    # Same points with alpha = 2 (alpha^2 = 4): id2 has 4 * 3.25 = 13 > 2.25
    # and survives; id1 has 4 * 1 = 4 <= 4 -> dominated (ties dominate).
    owner = _pad([(0, 0)])[0]
    cand = _pad([(1, 0), (2, 0), (0, 1.5)])
    ids, _ = oracle_mod.robust_prune_vectors(owner, cand, [0, 1, 2], R=8, alpha=2.0)
    assert ids.tolist() == [0, 2]
    # alpha = 0.5 (alpha^2 = 0.25): id1 has 0.25 * 1 <= 4 -> still dominated;
    # id2 has 0.25 * 3.25 = 0.8125 <= 2.25 -> dominated too.
    ids, _ = oracle_mod.robust_prune_vectors(owner, cand, [0, 1, 2], R=8, alpha=0.5)
    assert ids.tolist() == [0]


def test_degree_bound_cuts_the_sequence(oracle_mod):
    # Collinear points on opposite rays: (k, 0) and (-k, 0) for k = 1..4,
    # alpha = 1.  (1,0) dominates (2,0),(3,0),(4,0); (-1,0) dominates the rest
    # of its ray.  With R = 1 only the nearest (ties by id) remains.
    pts = [(1, 0), (2, 0), (3, 0), (4, 0), (-1, 0), (-2, 0), (-3, 0), (-4, 0)]
    owner = _pad([(0, 0)])[0]
    cand = _pad(pts)
    ids, _ = oracle_mod.robust_prune_vectors(owner, cand, list(range(8)), R=8, alpha=1.0)
    assert ids.tolist() == [0, 4]
    ids, _ = oracle_mod.robust_prune_vectors(owner, cand, list(range(8)), R=1, alpha=1.0)
    assert ids.tolist() == [0]


def test_no_domination_reduces_to_sort(oracle_mod):
    # alpha -> infinity: alpha^2 * d > rho for every d > 0, so nothing is ever
    # dominated and RobustPrune returns the R nearest by (rho, id), which a
    # library sort computes independently.  Integer inputs make rho exact.
    rng = np.random.default_rng(7)
    for trial in range(30):
        n, R, m = int(rng.integers(1, 80)), int(rng.integers(1, 40)), 16
        owner = rng.integers(0, 50, m).astype(np.float32)
        cand = rng.integers(0, 50, (n, m)).astype(np.float32)
        # distinct rows so that no pairwise distance is 0
        cand[:, 0] = np.arange(n)
        ids = rng.permutation(10_000)[:n].astype(np.uint32)
        got, rho = oracle_mod.robust_prune_vectors(owner, cand, ids, R=R, alpha=1e30)
        exact = ((cand.astype(np.int64) - owner.astype(np.int64)) ** 2).sum(1)
        order = np.lexsort((ids, exact))[:R]
        assert got.tolist() == ids[order].tolist()
        assert rho.tolist() == exact[order].astype(np.float64).tolist()


@pytest.mark.parametrize("alpha2", [1, 4])
def test_greedy_certificate_exact(oracle_mod, alpha2):
    # The rule's certificate, in exact integer arithmetic:
    #  (1) kept ids come out in ascending (rho, id);
    #  (2) no kept candidate is dominated by an earlier kept one;
    #  (3) every candidate ranked before the last kept one (or every candidate,
    #      if fewer than R were kept) that is not kept is dominated by an
    #      earlier kept one.
    rng = np.random.default_rng(8 + alpha2)
    alpha = math.sqrt(alpha2)
    for trial in range(40):
        n, R, m = int(rng.integers(2, 60)), int(rng.integers(1, 20)), 8
        owner = rng.integers(0, 20, m)
        cand = rng.integers(0, 20, (n, m))
        ids = np.arange(n, dtype=np.uint32) * 3 + 1
        got, _ = oracle_mod.robust_prune_vectors(owner.astype(np.float32), cand.astype(np.float32),
                                                 ids, R=R, alpha=alpha)
        rho = ((cand - owner) ** 2).sum(1)
        order = np.lexsort((ids, rho))
        pos = {int(ids[i]): r for r, i in enumerate(order)}
        kept_rows = [int((g - 1) // 3) for g in got]
        assert len(got) <= R
        assert [pos[int(g)] for g in got] == sorted(pos[int(g)] for g in got)

        def dominated(p_star, p):
            d = int(((cand[p_star] - cand[p]) ** 2).sum())
            return alpha2 * d <= int(rho[p])

        for a, b in itertools.combinations(range(len(kept_rows)), 2):
            assert not dominated(kept_rows[a], kept_rows[b])
        last = pos[int(got[-1])] if len(got) == R else n
        for r in range(last):
            i = int(order[r])
            if i in kept_rows:
                continue
            earlier = [k for k in kept_rows if pos[int(ids[k])] < r]
            assert any(dominated(k, i) for k in earlier), (trial, i)


def test_duplicates_collapse(oracle_mod):
    owner = _pad([(0, 0)])[0]
    cand = _pad([(1, 0), (1, 0), (0, 3)])
    ids, _ = oracle_mod.robust_prune_vectors(owner, cand, [5, 5, 9], R=8, alpha=1.0)
    assert ids.tolist() == [5, 9]
