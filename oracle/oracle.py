"""ctypes loader for the C oracle (test infrastructure only; see etale_oracle.c)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "etale_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
NIL = 0xFFFFFFFF

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fno-strict-aliasing", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Config(C.Structure):
    _fields_ = [("dim", C.c_uint32), ("metric", C.c_uint32), ("degree", C.c_uint32),
                ("capacity", C.c_uint64), ("build_beam", C.c_uint32), ("alpha", C.c_float),
                ("max_hops", C.c_uint32), ("max_cand", C.c_uint32), ("refine", C.c_uint32),
                ("max_batch", C.c_uint64), ("pool_slabs", C.c_uint64), ("n_entry", C.c_uint32)]


class _Stats(C.Structure):
    _fields_ = [("live", C.c_uint64), ("tombstones", C.c_uint64), ("reclaimed", C.c_uint64),
                ("next_id", C.c_uint64), ("pool", C.c_uint64), ("free_slabs", C.c_uint64),
                ("retired_slabs", C.c_uint64), ("used_slabs", C.c_uint64), ("n_entries", C.c_uint32),
                ("n_dist", C.c_uint64), ("n_expand", C.c_uint64), ("n_publish", C.c_uint64),
                ("n_prune", C.c_uint64), ("n_search", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.POINTER(_Config)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_dist.restype = C.c_float
        lib.orc_dist.argtypes = [P, P, C.c_uint32, C.c_uint32]
        lib.orc_dist64.restype = C.c_double
        lib.orc_dist64.argtypes = [P, P, C.c_uint32, C.c_uint32]
        lib.orc_robust_prune_vectors.restype = C.c_uint32
        lib.orc_robust_prune_vectors.argtypes = [P, P, P, C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_uint32, C.c_float, P, P]
        lib.orc_insert.restype = C.c_int
        lib.orc_insert.argtypes = [P, P, C.c_uint64, P]
        lib.orc_delete.restype = C.c_int
        lib.orc_delete.argtypes = [P, P, C.c_uint64, C.POINTER(C.c_uint64)]
        lib.orc_reclaim.restype = C.c_int
        lib.orc_reclaim.argtypes = [P]
        lib.orc_search.restype = C.c_int
        lib.orc_search.argtypes = [P, P, C.c_uint64, C.c_uint32, C.c_uint32, P, P]
        lib.orc_exact_knn.restype = C.c_int
        lib.orc_exact_knn.argtypes = [P, P, C.c_uint64, C.c_uint32, P, P]
        lib.orc_node.restype = C.c_int
        lib.orc_node.argtypes = [P, C.c_uint32, P, P, P, P]
        lib.orc_dump.argtypes = [P, P, P, P, P, P]
        lib.orc_get_stats.argtypes = [P, C.POINTER(_Stats)]
        lib.orc_effective_config.argtypes = [P, C.POINTER(_Config)]
        lib.orc_entries.restype = C.c_uint32
        lib.orc_entries.argtypes = [P, P]
        lib.orc_load.restype = P
        lib.orc_load.argtypes = [C.c_char_p, C.POINTER(_Config)]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def dist(a, b, metric: str = "l2") -> float:
    """Canonical fp32 distance (squared L2, or 1 - <a, b>)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_dist(_p(a), _p(b), a.size, 0 if metric == "l2" else 1))


def dist64(a, b, metric: str = "l2") -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_dist64(_p(a), _p(b), a.size, 0 if metric == "l2" else 1))


def robust_prune_vectors(owner, cand, ids, R: int, alpha: float, metric: str = "l2"):
    """RobustPrune on explicit vectors (no deletion flags)."""
    owner = np.ascontiguousarray(owner, dtype=np.float32)
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.empty(max(R, 1), np.uint32)
    rho = np.empty(max(R, 1), np.float32)
    n = _load().orc_robust_prune_vectors(_p(owner), _p(cand), _p(ids), ids.size, owner.size,
                                         0 if metric == "l2" else 1, R, alpha, _p(out), _p(rho))
    return out[:n].copy(), rho[:n].copy()


class Oracle:
    """One oracle index (deterministic-round semantics)."""

    def __init__(self, dim: int, metric: str, degree: int, capacity: int, *,
                 build_beam: int = 64, alpha: float = 1.2, max_hops: int = 0,
                 max_cand: int = 0, refine: int = 1, max_batch: int = 0, pool_slabs: int = 0,
                 n_entry: int = 0):
        self.lib = _load()
        cfg = _Config(dim, 0 if metric == "l2" else 1, degree, capacity, build_beam, alpha,
                      max_hops, max_cand, refine, max_batch, pool_slabs, n_entry)
        self.h = self.lib.orc_create(C.byref(cfg))
        if not self.h:
            raise ValueError("orc_create rejected the configuration")
        self.dim, self.degree, self.capacity = dim, degree, capacity
        self.metric = metric

    @classmethod
    def load(cls, path: str, capacity: int = 0, *, build_beam: int = 64, alpha: float = 1.2,
             max_hops: int = 0, max_cand: int = 0, refine: int = 1, max_batch: int = 0,
             pool_slabs: int = 0, n_entry: int = 0) -> "Oracle":
        """orc_load: an oracle index rebuilt from a snapshot file (dim, metric and
        degree from the file; the maintenance knobs from the arguments)."""
        lib = _load()
        cfg = _Config(0, 0, 0, capacity, build_beam, alpha, max_hops, max_cand, refine, max_batch,
                      pool_slabs, n_entry)
        h = lib.orc_load(os.fsencode(path), C.byref(cfg))
        if not h:
            raise ValueError(f"orc_load could not read {path}")
        self = cls.__new__(cls)
        self.lib, self.h = lib, h
        c = self.config()
        self.dim, self.degree, self.capacity = c["dim"], c["degree"], c["capacity"]
        self.metric = "l2" if c["metric"] == 0 else "ip"
        return self

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    def config(self) -> dict:
        c = _Config()
        self.lib.orc_effective_config(self.h, C.byref(c))
        return {f: getattr(c, f) for f, _ in _Config._fields_}

    def insert(self, vecs: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(vecs, dtype=np.float32).reshape(-1, self.dim)
        ids = np.empty(v.shape[0], np.uint32)
        st = self.lib.orc_insert(self.h, _p(v), v.shape[0], _p(ids))
        if st:
            raise RuntimeError(f"orc_insert status {st}")
        return ids

    def delete(self, ids) -> int:
        d = np.ascontiguousarray(ids, dtype=np.uint32)
        n = C.c_uint64(0)
        st = self.lib.orc_delete(self.h, _p(d), d.size, C.byref(n))
        if st:
            raise RuntimeError(f"orc_delete status {st}")
        return int(n.value)

    def reclaim(self) -> None:
        st = self.lib.orc_reclaim(self.h)
        if st:
            raise RuntimeError(f"orc_reclaim status {st}")

    def search(self, q: np.ndarray, k: int, beam: int):
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, self.dim)
        ids = np.empty((q.shape[0], k), np.uint32)
        d = np.empty((q.shape[0], k), np.float32)
        self.lib.orc_search(self.h, _p(q), q.shape[0], k, beam, _p(ids), _p(d))
        return ids, d

    def exact_knn(self, q: np.ndarray, k: int):
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, self.dim)
        ids = np.empty((q.shape[0], k), np.uint32)
        d = np.empty((q.shape[0], k), np.float64)
        self.lib.orc_exact_knn(self.h, _p(q), q.shape[0], k, _p(ids), _p(d))
        return ids, d

    def node(self, u: int):
        R = self.degree
        ids = np.empty(R, np.uint32)
        rho = np.empty(R, np.float32)
        de, hs = C.c_uint32(0), C.c_uint32(0)
        n = self.lib.orc_node(self.h, u, C.byref(de), C.byref(hs), _p(ids), _p(rho))
        return int(de.value), bool(hs.value), ids[:n].copy(), rho[:n].copy()

    def dump(self):
        """Logical graph over ids [0, next_id): (del, has_slab, deg, ids[n,R], rho[n,R])."""
        n = self.stats()["next_id"]
        R = self.degree
        de = np.empty(n, np.uint8)
        hs = np.empty(n, np.uint8)
        dg = np.empty(n, np.uint8)
        ids = np.empty((n, R), np.uint32)
        rho = np.empty((n, R), np.float32)
        if n:
            self.lib.orc_dump(self.h, _p(de), _p(hs), _p(dg), _p(ids), _p(rho))
        return de, hs, dg, ids, rho

    def entries(self) -> np.ndarray:
        out = np.empty(self.config()["n_entry"], np.uint32)
        n = self.lib.orc_entries(self.h, _p(out))
        return out[:n].copy()

    def stats(self) -> dict:
        s = _Stats()
        self.lib.orc_get_stats(self.h, C.byref(s))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}
