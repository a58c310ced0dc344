"""Snapshot files on CPU: the oracle's reader (orc_load) rebuilds exactly the
state a file describes.  The file is written by tests/snapshot_io.py from an
oracle's own state (Definition 1: vectors, reference words, slab lists), so
after loading, the two oracles must hold the same logical graph and entry
set, answer the same searches, and stay equal through further churn rounds
(Algorithms 2-4)."""
import numpy as np
import pytest

from paper_2607_02543_gb300 import workloads as W
from tests import snapshot_io

KNOBS = dict(build_beam=32, refine=2, n_entry=64)


def _same_dump(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))


def _snapshot_of(o, vectors, path):
    snapshot_io.write(path, dim=o.dim, metric=o.metric, degree=o.degree, capacity=o.capacity,
                      vectors=vectors, dump=o.dump(), entries=o.entries())


def test_oracle_load_round_trip(oracle_mod, tmp_path):
    w = W.scaled(W.SMALL, 800, n_queries=100, rounds=3)
    p = W.make_plan(w)
    X = np.concatenate([p.base] + p.inserts)
    o = oracle_mod.Oracle(w.dim, "l2", w.degree, w.capacity, **KNOBS)
    o.insert(p.base)
    rng = np.random.default_rng(1)
    o.delete(rng.choice(w.n_base, 40, replace=False).astype(np.uint32))   # tombstones, no reclaim
    path = str(tmp_path / "o.snap")
    _snapshot_of(o, X, path)
    o2 = oracle_mod.Oracle.load(path, **KNOBS)
    _same_dump(o.dump(), o2.dump())
    assert np.array_equal(o.entries(), o2.entries())
    s1, s2 = o.stats(), o2.stats()
    for key in ("live", "tombstones", "reclaimed", "next_id", "used_slabs"):
        assert s1[key] == s2[key], key
    a, b = o.search(p.queries, 10, 48), o2.search(p.queries, 10, 48)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    for r in range(w.rounds):
        for g in (o, o2):
            g.reclaim()
            g.delete(np.arange(r * 50, r * 50 + 25, dtype=np.uint32))
            g.insert(p.inserts[r])
        _same_dump(o.dump(), o2.dump())
    a, b = o.search(p.queries, 10, 48), o2.search(p.queries, 10, 48)
    assert np.array_equal(a[0], b[0])


def test_oracle_load_rejects_malformed(oracle_mod, tmp_path):
    w = W.scaled(W.SMALL, 200, n_queries=10, rounds=1)
    p = W.make_plan(w)
    o = oracle_mod.Oracle(w.dim, "l2", w.degree, w.capacity, **KNOBS)
    o.insert(p.base)
    good = str(tmp_path / "good.snap")
    _snapshot_of(o, p.base, good)
    raw = open(good, "rb").read()
    cases = {"magic": b"XTALESN1" + raw[8:], "truncated": raw[:-7]}
    # an out-of-range neighbour id inside the first list
    d = snapshot_io.read(good)
    off = 48 + 8 * 17 + 4 * d["x"].size + 2 * d["x"].shape[0]
    bad_id = bytearray(raw)
    bad_id[off:off + 4] = (10 ** 6).to_bytes(4, "little")
    cases["id"] = bytes(bad_id)
    for name, data in cases.items():
        path = str(tmp_path / f"{name}.snap")
        open(path, "wb").write(data)
        with pytest.raises(ValueError):
            oracle_mod.Oracle.load(path, **KNOBS)


def test_writer_reader_agree(oracle_mod, tmp_path):
    w = W.scaled(W.SMALL, 150, n_queries=10, rounds=1)
    p = W.make_plan(w)
    o = oracle_mod.Oracle(w.dim, "l2", w.degree, w.capacity, **KNOBS)
    o.insert(p.base)
    o.delete(np.arange(0, 150, 7, dtype=np.uint32))
    path = str(tmp_path / "w.snap")
    _snapshot_of(o, p.base, path)
    d = snapshot_io.read(path)
    de, hs, dg, ids, rho = o.dump()
    assert np.array_equal(d["deleted"], de) and np.array_equal(d["has_slab"], hs)
    assert np.array_equal(d["deg"], dg)
    mask = np.arange(w.degree)[None, :] < dg[:, None]
    assert np.array_equal(d["ids"][mask], ids[mask])
    assert np.array_equal(d["rho"][mask].view(np.uint32), rho[mask].view(np.uint32))
    assert np.array_equal(d["x"], p.base) and np.array_equal(d["entries"], o.entries())
