"""Invariant checks on a dumped logical graph (shared by oracle and GPU tests).

A dump is (del, has_slab, deg, ids[n, R], rho[n, R]) over ids [0, n).  The
checks restate the paper's invariants:
  degree <= R (Definition 1); no self loop or repeated neighbour; slabs in
  (rho, id) order; rho equal to the canonical distance to the owner;
  no live node points at a reclaimed id (Proposition 2);
  after Reclaim: no live -> tombstone edge and no tombstone left
  (Algorithm 4, Proposition 3).
"""
from __future__ import annotations

import numpy as np

NIL = 0xFFFFFFFF


def order_key(rho: np.ndarray, ids: np.ndarray) -> np.ndarray:
    u = rho.astype(np.float32).view(np.uint32).astype(np.uint64)
    neg = (u & 0x80000000) != 0
    u = np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000)
    return (u << np.uint64(32)) | ids.astype(np.uint64)


def check_graph(dump, R: int, *, after_reclaim: bool = False, vectors=None, dist=None,
                sample: int | None = None, rng=None) -> dict:
    de, hs, dg, ids, rho = dump
    n = de.shape[0]
    assert (dg <= R).all(), "degree above R"
    live = (de == 0) & (hs == 1)
    tomb = (de == 1) & (hs == 1)
    reclaimed = (de == 1) & (hs == 0)
    assert (dg[hs == 0] == 0).all()
    rows = np.nonzero(hs)[0]
    for u in rows:
        d = int(dg[u])
        nb = ids[u, :d]
        assert (nb < n).all(), f"node {u}: neighbour id out of range"
        assert (nb != u).all(), f"node {u}: self loop"
        assert np.unique(nb).size == d, f"node {u}: repeated neighbour"
        if d > 1:
            k = order_key(rho[u, :d], nb)
            assert (k[1:] > k[:-1]).all(), \
                f"node {u}: slab not in (rho, id) order"
    # no live node points at a reclaimed id
    lr = np.nonzero(live)[0]
    if lr.size:
        mask = np.arange(R)[None, :] < dg[lr, None]
        tgt = ids[lr][mask]
        assert not reclaimed[tgt].any(), "live node points at a reclaimed id"
        if after_reclaim:
            assert not (de[tgt] == 1).any(), "live -> tombstone edge after reclaim"
    if after_reclaim:
        assert tomb.sum() == 0, "tombstone left after reclaim"
    if vectors is not None and dist is not None:
        cand = rows if sample is None else (rng or np.random.default_rng(0)).choice(
            rows, size=min(sample, rows.size), replace=False)
        for u in cand:
            for j in range(int(dg[u])):
                a = int(ids[u, j])
                assert dist(vectors[u], vectors[a]) == float(rho[u, j]), \
                    f"rho of edge {u}->{a} is not the canonical distance"
    return {"live": int(live.sum()), "tombstones": int(tomb.sum()),
            "reclaimed": int(reclaimed.sum()), "mean_degree": float(dg[live].mean()) if live.any() else 0.0}


def reachable_from(dump, sources) -> np.ndarray:
    """Ids reached by following slabs from the sources (tombstones relay)."""
    de, hs, dg, ids, _ = dump
    n = de.shape[0]
    seen = np.zeros(n, bool)
    stack = [int(s) for s in sources]
    for s in stack:
        seen[s] = True
    while stack:
        u = stack.pop()
        if not hs[u]:
            continue
        for a in ids[u, :int(dg[u])]:
            a = int(a)
            if not seen[a]:
                seen[a] = True
                stack.append(a)
    return seen


def recall_at_k(found: np.ndarray, truth: np.ndarray) -> float:
    k = truth.shape[1]
    hits = 0
    for f, t in zip(found, truth):
        hits += len(set(f.tolist()) & set(t.tolist()) - {NIL})
    return hits / (truth.shape[0] * k)
