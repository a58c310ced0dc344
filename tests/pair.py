"""Helpers that drive the CUDA index (through the C ABI) and the oracle side
by side on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from paper_2607_02543_gb300 import workloads as W

# oracle refine numbering: 0 off, 1 two-hop, 2 peers; C ABI: "off", "peers"
ORACLE_REFINE = {"off": 0, "peers": 2}


def make_pair(oracle_mod, dim, metric, degree, capacity, *, build_beam=64, alpha=1.2, refine="peers",
              max_batch=0, n_entry=0, mode="deterministic", max_cand=0, max_hops=0, with_oracle=True,
              gram="default", stage_kb=0):
    from paper_2607_02543_gb300 import Index
    g = Index(dim, metric, degree, capacity, build_beam=build_beam, alpha=alpha, refine=refine,
              max_batch=max_batch, n_entry=n_entry, mode=mode, max_cand=max_cand, max_hops=max_hops,
              gram=gram, stage_kb=stage_kb)
    o = None
    if with_oracle:
        o = oracle_mod.Oracle(dim, metric, degree, capacity, build_beam=build_beam, alpha=alpha,
                              refine=ORACLE_REFINE[refine], max_batch=max_batch, n_entry=n_entry,
                              max_cand=max_cand, max_hops=max_hops)
    return g, o


def graphs_equal(gd, od, R):
    """Bit-exact comparison of two logical graphs; returns a list of problems."""
    problems = []
    names = ("deleted", "has_slab", "degree")
    for name, a, b in zip(names, gd[:3], od[:3]):
        if a.shape != b.shape:
            return [f"{name}: shape {a.shape} vs {b.shape}"]
        bad = np.nonzero(a != b)[0]
        if bad.size:
            problems.append(f"{name} differs at {bad.size} ids, first {bad[:5].tolist()}")
    deg = gd[2]
    mask = np.arange(R)[None, :] < deg[:, None]
    ids_bad = np.nonzero(((gd[3] != od[3]) & mask).any(1))[0]
    if ids_bad.size:
        u = int(ids_bad[0])
        problems.append(f"neighbour ids differ at {ids_bad.size} nodes, first {u}: "
                        f"gpu {gd[3][u, :deg[u]].tolist()} oracle {od[3][u, :deg[u]].tolist()}")
    rho_bad = np.nonzero(((gd[4].view(np.uint32) != od[4].view(np.uint32)) & mask).any(1))[0]
    if rho_bad.size:
        problems.append(f"rho bits differ at {rho_bad.size} nodes, first {int(rho_bad[0])}")
    return problems


def churn_round(g, o, plan, r, n_delete, rng_state=None, reclaim=True):
    """One round: delete n_delete uniformly chosen live ids, insert the round's
    vectors, reclaim.  The delete choice comes from the oracle side's live set
    when present (the two are equal in deterministic mode), else the GPU's."""
    de = (o.dump()[0] if o is not None else g.export_graph()[0])
    hs = (o.dump()[1] if o is not None else g.export_graph()[1])
    live = np.nonzero((de == 0) & (hs == 1))[0].astype(np.uint32)
    dele = W.choose_deletes(plan.delete_rng, live, n_delete)
    ng = g.delete(dele)
    no = o.delete(dele) if o is not None else ng
    gi = g.insert(plan.inserts[r])
    oi = o.insert(plan.inserts[r]) if o is not None else gi
    if reclaim:
        g.reclaim()
        if o is not None:
            o.reclaim()
    return dele, ng, no, gi, oi
