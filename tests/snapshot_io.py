"""Writer and reader of the snapshot file format declared in include/etale.h
(version 1), in plain numpy, for tests: they write an oracle's state into a
file both loaders read, and check what the library writes."""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"ETALESN1"
N_CFG = 17


def write(path, *, dim, metric, degree, capacity, vectors, dump, entries, cfg_words=None):
    """dump = (deleted, has_slab, degree, ids[n, R], rho[n, R]) over ids [0, n)."""
    de, hs, dg, ids, rho = dump
    n = de.shape[0]
    cfg = np.zeros(N_CFG, np.uint64) if cfg_words is None else np.asarray(cfg_words, np.uint64)
    entries = np.asarray(entries, np.uint32)
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<4I", 1, dim, 0 if metric == "l2" else 1, degree))
        f.write(struct.pack("<2Q", capacity, n))
        f.write(struct.pack("<2I", entries.size, N_CFG))
        f.write(cfg.astype("<u8").tobytes())
        f.write(np.ascontiguousarray(vectors[:n], dtype="<f4").tobytes())
        flags = (de.astype(np.uint8) & 1) | ((hs.astype(np.uint8) & 1) << 1)
        f.write(flags.tobytes())
        f.write(np.where(hs == 1, dg, 0).astype(np.uint8).tobytes())
        for u in range(n):
            if hs[u]:
                rec = np.empty(int(dg[u]), dtype=[("id", "<u4"), ("rho", "<f4")])
                rec["id"], rec["rho"] = ids[u, :dg[u]], rho[u, :dg[u]]
                f.write(rec.tobytes())
        f.write(entries.astype("<u4").tobytes())


def read(path):
    """The file's contents as a dict (dump in the same layout as write's)."""
    with open(path, "rb") as f:
        b = f.read()
    assert b[:8] == MAGIC
    ver, dim, metric, R = struct.unpack_from("<4I", b, 8)
    capacity, n = struct.unpack_from("<2Q", b, 24)
    ne, ncfg = struct.unpack_from("<2I", b, 40)
    off = 48
    cfg = np.frombuffer(b, "<u8", ncfg, off); off += 8 * ncfg
    x = np.frombuffer(b, "<f4", n * dim, off).reshape(n, dim); off += 4 * n * dim
    flags = np.frombuffer(b, np.uint8, n, off); off += n
    dg = np.frombuffer(b, np.uint8, n, off).copy(); off += n
    ids = np.full((n, R), 0xFFFFFFFF, np.uint32)
    rho = np.zeros((n, R), np.float32)
    for u in range(n):
        if flags[u] & 2:
            rec = np.frombuffer(b, [("id", "<u4"), ("rho", "<f4")], int(dg[u]), off)
            ids[u, :dg[u]], rho[u, :dg[u]] = rec["id"], rec["rho"]
            off += 8 * int(dg[u])
    entries = np.frombuffer(b, "<u4", ne, off).copy(); off += 4 * ne
    assert off == len(b), (off, len(b))
    return {"version": ver, "dim": dim, "metric": metric, "degree": R, "capacity": capacity, "cfg": cfg,
            "x": x, "deleted": flags & 1, "has_slab": (flags >> 1) & 1, "hint": (flags >> 2) & 1,
            "deg": dg, "ids": ids, "rho": rho, "entries": entries}
