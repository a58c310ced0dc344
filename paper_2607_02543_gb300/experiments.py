"""Measurements beyond the headline churn round, run on the GPU index.

- reclaim_interval (Proposition 4, Remark 1): reclaim cost and dirty-node
  count after t accumulated tombstones, the saturating fit
  M (1 - exp(-t / tau)), and the uniform model's prediction.
- deletion_stress (pure deletions): delete 10% of the live set per round,
  reclaim, until half of it is gone; recall, footprint and reclaim cost.
- concurrent_latency (two streams, Sec. 5.5): query-batch latency alone and
  while a writer churns the index on another stream, with recall on an anchor
  query set whose exact neighbours never change.

The host-side helpers (model, fit, edge counts) are plain numpy and are
tested on the CPU; the run_* functions need a GPU.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import workloads as W


# ---- Proposition 4's uniform model -------------------------------------------
def dirty_model(L: float, dbar: float, t) -> np.ndarray:
    """Expected dirty nodes after t tombstones when each strands dbar in-edges
    on live nodes drawn independently and uniformly from L."""
    t = np.asarray(t, dtype=np.float64)
    return L * (1.0 - np.exp(dbar * t * np.log1p(-1.0 / L)))


def dirty_monte_carlo(L: int, dbar: float, t: int, rng: np.random.Generator) -> int:
    """One draw of the same model: distinct nodes hit by round(dbar * t) edges."""
    hits = rng.integers(0, L, size=int(round(dbar * t)))
    return int(np.unique(hits).size)


def fit_saturating(t, y) -> dict:
    """Least-squares fit of y = M (1 - exp(-t / tau)); returns M, tau and R^2."""
    from scipy.optimize import curve_fit
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)

    def f(x, M, tau):
        return M * (1.0 - np.exp(-x / tau))

    p0 = (max(float(y.max()) * 1.5, 1e-9), max(float(np.median(t)), 1.0))
    (M, tau), _ = curve_fit(f, t, y, p0=p0, maxfev=20000)
    res = y - f(t, M, tau)
    ss_tot = float(((y - y.mean()) ** 2).sum())
    r2 = 1.0 - float((res ** 2).sum()) / ss_tot if ss_tot > 0 else 1.0
    return {"M": float(M), "tau": float(tau), "r2": r2}


def dead_edge_counts(graph) -> dict:
    """From an exported graph (deleted, has_slab, degree, ids, rho): live nodes,
    edges out of live nodes, edges from live nodes into tombstones (dead
    edges) and live nodes with at least one (dirty)."""
    deleted, has_slab, degree, ids = graph[0], graph[1], graph[2], graph[3]
    n, R = ids.shape
    live = (deleted == 0) & (has_slab == 1)
    mask = np.arange(R)[None, :] < degree[:, None]
    tgt = np.where(mask, ids, 0).astype(np.int64)
    tomb = (deleted == 1) & (has_slab == 1)
    dead = mask & tomb[np.minimum(tgt, n - 1)] & (tgt < n)
    dead &= live[:, None]
    return {"live": int(live.sum()), "live_edges": int((mask & live[:, None]).sum()),
            "dead_edges": int(dead.sum()), "dirty": int(dead.any(axis=1).sum())}


def _recall(got: np.ndarray, gt: np.ndarray, k: int) -> float:
    return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(got, gt)]))


def _build(w: W.Workload, capacity: int, mode: str = "lockfree", n_entry: int = 4096, max_cand: int = 64):
    import torch
    from . import Index
    plan = W.make_plan(W.dataclasses.replace(w, rounds=0))
    idx = Index(w.dim, w.metric, w.degree, capacity, build_beam=w.build_beam, mode=mode, n_entry=n_entry,
                max_cand=max_cand)
    idx.insert(torch.from_numpy(plan.base).cuda())
    idx.reclaim()
    torch.cuda.synchronize()
    return idx, plan


# ---- f1: reclaim interval ----------------------------------------------------
def run_reclaim_interval(w: W.Workload, rounds=(1, 2, 4, 8, 12, 16, 24, 32)) -> dict:
    """Tombstones accumulate over churn rounds with no Reclaim in between (each
    round: 1% of the live set deleted uniformly, as many fresh rows inserted),
    as when reclamation is deferred.  For each T in `rounds` a fresh index is
    built and churned T rounds; then dead edges (live -> tombstone) and dirty
    nodes (live nodes with one) are counted from the exported graph, and one
    Reclaim is timed (CUDA events) with the republications it makes, which
    equal the dirty-node count.  t = tombstones accumulated."""
    import torch
    mix = W.Mixture(w)
    n_ch = max(1, w.n_base // 100)
    fresh = mix.draw("inserts", n_ch * max(rounds))
    pts = []
    for T in rounds:
        idx, _ = _build(w, w.n_base + n_ch * max(rounds) + 10)
        rng = np.random.default_rng(w.seed + 1)
        alive = np.zeros(w.n_base + n_ch * max(rounds) + 10, bool)
        alive[:w.n_base] = True
        for r in range(T):
            dele = rng.choice(np.nonzero(alive)[0], size=n_ch, replace=False).astype(np.uint32)
            idx.delete(dele)
            alive[dele] = False
            alive[idx.insert(fresh[r * n_ch:(r + 1) * n_ch])] = True
        torch.cuda.synchronize()
        counts = dead_edge_counts(idx.export_graph())
        s0 = idx.stats()
        idx.set_profiling(True)
        idx.profile(reset=True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        idx.reclaim(st)
        e1.record(st)
        torch.cuda.synchronize()
        prof = idx.profile(reset=True)
        s1 = idx.stats()
        pts.append({"rounds": T, "t": int(s0["tombstones"]), "reclaim_ms": e0.elapsed_time(e1),
                    "compact_ms": prof["compact"][0], "republished": int(s1["n_publish"] - s0["n_publish"]),
                    "dirty": counts["dirty"], "dead_edges": counts["dead_edges"], "live": counts["live"],
                    "mean_in_degree": counts["live_edges"] / max(1, counts["live"])})
        del idx
        torch.cuda.empty_cache()
    L = float(np.mean([p["live"] for p in pts]))
    dbar = float(np.mean([p["mean_in_degree"] for p in pts]))
    ts = np.array([p["t"] for p in pts], dtype=np.float64)
    mc_rng = np.random.default_rng(7)
    for p in pts:
        p["model_dirty"] = float(dirty_model(p["live"], p["mean_in_degree"], p["t"]))
        p["monte_carlo_dirty"] = dirty_monte_carlo(int(p["live"]), p["mean_in_degree"], p["t"], mc_rng)
    return {"experiment": "reclaim_interval", "workload": w.name, "churn_per_round": n_ch, "points": pts,
            "fit_dirty": fit_saturating(ts, [p["dirty"] for p in pts]),
            "fit_reclaim_ms": fit_saturating(ts, [p["reclaim_ms"] for p in pts]),
            "fit_dead_edges_linear_slope": float(np.polyfit(ts, [p["dead_edges"] for p in pts], 1)[0]),
            "model_tau": L / dbar, "L": L, "mean_in_degree": dbar}


# ---- f2: pure deletion stress ------------------------------------------------
def run_deletion_stress(w: W.Workload, frac: float = 0.10, beam: int = 128) -> dict:
    """Delete frac of the live set per round (uniformly), then Reclaim, until at
    most half of the build remains.  Per round: delete and reclaim time,
    Recall@10 of the query set against the exact top-10 of the live set, used
    slabs and device bytes of the live index."""
    import torch
    idx, plan = _build(w, w.n_base + 10)
    d_q = torch.from_numpy(plan.queries).cuda()
    rng = np.random.default_rng(w.seed + 2)
    rows, live0 = [], w.n_base
    row_bytes = w.dim * 4 + 8
    while True:
        s = idx.stats()
        if s["live"] <= live0 // 2:
            break
        g = idx.export_graph()
        live_ids = np.nonzero((g[0] == 0) & (g[1] == 1))[0].astype(np.uint32)
        dele = rng.choice(live_ids, size=int(frac * live_ids.size), replace=False).astype(np.uint32)
        st = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(st)
        idx.delete(dele, st)
        ev[1].record(st)
        idx.reclaim(st)
        ev[2].record(st)
        torch.cuda.synchronize()
        gt, _ = idx.ground_truth(d_q, w.k)
        ids, _ = idx.search(d_q, w.k, beam)
        s = idx.stats()
        rows.append({"live": int(s["live"]), "deleted": int(dele.size), "delete_ms": ev[0].elapsed_time(ev[1]),
                     "reclaim_ms": ev[1].elapsed_time(ev[2]),
                     "recall_at_10": _recall(ids.cpu().numpy().view(np.uint32), gt.cpu().numpy().view(np.uint32),
                                             w.k),
                     "used_slabs": int(s["used_slabs"]),
                     "index_bytes": int(s["live"]) * row_bytes + int(s["used_slabs"]) * 8 * w.degree})
    return {"experiment": "deletion_stress", "workload": w.name, "fraction_per_round": frac, "beam": beam,
            "rounds": rows}


# ---- f3: concurrent query-vs-update latency ----------------------------------
def run_concurrent_latency(w: W.Workload, batch: int = 1000, n_batches: int = 2000, beam: int = 128,
                           extra: int = 4_000_000, n_fresh: int = 2_000_000) -> dict:
    """Latency of 1,000-query batches alone and while a writer thread churns the
    index (0.05% deletes + 0.05% inserts + Reclaim per round) on its own stream, in
    concurrent mode.  The anchor queries' exact top-10 never changes: deletes
    skip those ids, and inserts come from the same mixture shifted far from
    every anchor (+10^4 on each coordinate)."""
    import torch
    idx, plan = _build(w, w.n_base + extra)
    anchors = plan.queries[:batch]
    d_a = torch.from_numpy(anchors).cuda()
    gt, _ = idx.ground_truth(d_a, w.k)
    gt_np = gt.cpu().numpy().view(np.uint32)
    protected = np.unique(gt_np)
    mix = W.Mixture(w)
    fresh = (mix.draw("inserts", n_fresh) + 1.0e4).astype(np.float32)
    qs, us = torch.cuda.Stream(), torch.cuda.Stream()

    def batches(n):
        lat, rec = [], []
        out_ids = torch.empty((batch, w.k), dtype=torch.int32, device="cuda")
        out_d = torch.empty((batch, w.k), dtype=torch.float32, device="cuda")
        for i in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(qs)
            idx.search(d_a, w.k, beam, qs, out=(out_ids, out_d))
            e1.record(qs)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
            if i % 10 == 0:   # recall of every tenth batch (host-side set work)
                rec.append(_recall(out_ids.cpu().numpy().view(np.uint32), gt_np, w.k))
        return lat, rec

    def pct(a):
        a = np.asarray(a)
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "mean_ms": float(a.mean())}

    batches(5)
    q_lat, q_rec = batches(n_batches)
    idx.set_concurrent(True)
    stop = threading.Event()
    rounds = [0]
    rng = np.random.default_rng(w.seed + 3)
    alive = np.zeros(w.n_base + extra, bool)
    alive[:w.n_base] = True
    keep = np.zeros_like(alive)
    keep[protected] = True

    errors = []

    def writer():
        try:
            write_rounds()
        except Exception as e:   # surfaced after join: a failed writer fails the run
            errors.append(e)
            stop.set()

    def write_rounds():
        # the live set is tracked on the host from the ids each call returns;
        # 0.05% of the build per round keeps the live set's make-up steady
        # over the measured window
        off = 0
        n_ch = max(1, w.n_base // 2000)
        while not stop.is_set() and off + n_ch <= len(fresh):
            cand = np.nonzero(alive & ~keep)[0].astype(np.uint32)
            dele = rng.choice(cand, size=n_ch, replace=False).astype(np.uint32)
            idx.delete(dele, us)
            alive[dele] = False
            alive[idx.insert(fresh[off:off + n_ch], us)] = True
            idx.reclaim(us)
            us.synchronize()
            off += n_ch
            rounds[0] += 1

    th = threading.Thread(target=writer)
    th.start()
    time.sleep(0.5)
    c_lat, c_rec = batches(n_batches)
    stop.set()
    th.join()
    idx.set_concurrent(False)
    if errors:
        raise errors[0]
    return {"experiment": "concurrent_latency", "workload": w.name, "batch": batch, "beam": beam,
            "quiescent": {**pct(q_lat), "recall_at_10": float(np.mean(q_rec))},
            "concurrent": {**pct(c_lat), "recall_at_10": float(np.mean(c_rec)), "writer_rounds": rounds[0],
                           "churned_fraction": rounds[0] * max(1, w.n_base // 2000) / w.n_base}}
