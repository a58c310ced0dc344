"""Thin ctypes binding of include/etale.h (argument marshalling only).

Every step of the index runs in libetale.so on the GPU.  There is no CPU
fallback: loading fails loudly when the library has not been built or no CUDA
device is present.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libetale.so")
NIL = 0xFFFFFFFF

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECAPACITY", 4: "ECUDA", 5: "ETIMEOUT", 6: "EINTERNAL"}
MODES = {"deterministic": 0, "lockfree": 1}
REFINE = {"default": 0, "off": 1, "peers": 2}


class EtaleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("build_beam", C.c_uint32), ("alpha", C.c_float), ("max_hops", C.c_uint32),
                ("max_cand", C.c_uint32), ("refine", C.c_uint32), ("max_batch", C.c_uint64),
                ("pool_slabs", C.c_uint64), ("n_entry", C.c_uint32), ("mode", C.c_uint32),
                ("cas_budget", C.c_uint32), ("stage_kb", C.c_uint32), ("gram", C.c_uint32),
                ("copies", C.c_uint32), ("rerank", C.c_uint32), ("gt", C.c_uint32),
                ("seed", C.c_uint32), ("exact_rows", C.c_uint32)]


class Tuning(C.Structure):
    _fields_ = [("stage_rows", C.c_uint32), ("seen_bits", C.c_uint32), ("ms", C.c_float),
                ("warps_per_block", C.c_uint32), ("keys_tc", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("live", C.c_uint64), ("tombstones", C.c_uint64), ("reclaimed", C.c_uint64),
                ("next_id", C.c_uint64), ("capacity", C.c_uint64), ("pool_slabs", C.c_uint64),
                ("free_slabs", C.c_uint64), ("retired_slabs", C.c_uint64), ("used_slabs", C.c_uint64),
                ("n_entries", C.c_uint32), ("degree", C.c_uint32), ("n_publish", C.c_uint64),
                ("n_cas_retry", C.c_uint64), ("n_dropped", C.c_uint64), ("n_expand", C.c_uint64),
                ("n_dist", C.c_uint64), ("device_bytes", C.c_uint64), ("exact_rows", C.c_uint64),
                ("dim", C.c_uint32), ("metric", C.c_uint32)]


EXPORTS = ["etale_config_default", "etale_create", "etale_destroy", "etale_insert", "etale_delete",
           "etale_reclaim", "etale_search", "etale_ground_truth", "etale_export_graph",
           "etale_get_entries", "etale_stats", "etale_get_config", "etale_last_error",
           "etale_kernel_launches", "etale_set_profiling", "etale_get_profile", "etale_search_static",
           "etale_set_search_precision", "etale_export_copies", "etale_set_concurrent",
           "etale_set_search_tuning", "etale_set_search_keys", "etale_autotune_search", "etale_search_graph_create",
           "etale_search_graph_launch", "etale_search_graph_check", "etale_search_graph_destroy",
           "etale_selftest_bounded_wait", "etale_ground_truth_info", "etale_set_exact_rows", "etale_save",
           "etale_load", "etale_search_eval_count", "etale_round_graph_create",
           "etale_round_graph_launch", "etale_round_graph_sync", "etale_round_graph_destroy",
           "etale_set_insert_precision", "etale_set_rerank", "etale_autotune_beam", "etale_ring_create",
           "etale_ring_buffers", "etale_ring_publish", "etale_ring_close", "etale_ring_launch", "etale_ring_destroy", "etale_ring_serve", "etale_set_writer_share", "etale_get_work", "etale_ring_stats"]
PHASES = ["seed", "search_insert", "prune", "offer_sort", "offer_fold", "refine", "delete_prep",
          "repair_k", "repair_fold", "entries", "compact", "reclaim", "search_query", "recycle",
          "gt_prep", "gt_tensor", "gt_merge", "gt_exact"]
# etale_get_work kinds, in the header's order; each is timed as the phase named
WORK_KINDS = ["prune", "offer_fold", "refine", "repair_k", "repair_fold", "compact"]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libetale.so and declare every entry point.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2607_02543_gb300.build.build()")
        lib = C.CDLL(path)
        P, U32, U64 = C.c_void_p, C.c_uint32, C.c_uint64
        sig = {
            "etale_config_default": ([C.POINTER(Config)], C.c_int),
            "etale_create": ([U32, C.c_int, U32, U64, C.POINTER(Config), C.POINTER(P)], C.c_int),
            "etale_destroy": ([P], C.c_int),
            "etale_insert": ([P, P, U64, P, P], C.c_int),
            "etale_delete": ([P, P, U64, C.POINTER(U64), P], C.c_int),
            "etale_reclaim": ([P, P], C.c_int),
            "etale_search": ([P, P, U64, U32, U32, P, P, P], C.c_int),
            "etale_ground_truth": ([P, P, U64, U32, P, P, P], C.c_int),
            "etale_export_graph": ([P, U64, P, P, P, P, P, P], C.c_int),
            "etale_get_entries": ([P, P, C.POINTER(U32)], C.c_int),
            "etale_stats": ([P, C.POINTER(Stats)], C.c_int),
            "etale_get_config": ([P, C.POINTER(Config)], C.c_int),
            "etale_last_error": ([P], C.c_char_p),
            "etale_kernel_launches": ([P], U64),
            "etale_set_profiling": ([P, C.c_int], C.c_int),
            "etale_get_profile": ([P, P, P, U32, C.c_int], C.c_int),
            "etale_search_static": ([P, P, U64, U32, U32, P, P, P], C.c_int),
            "etale_set_search_precision": ([P, C.c_int], C.c_int),
            "etale_set_insert_precision": ([P, C.c_int], C.c_int),
            "etale_set_rerank": ([P, U32], C.c_int),
            "etale_set_writer_share": ([P, C.c_float], C.c_int),
            "etale_get_work": ([P, P, P, U32, C.c_int], C.c_int),
            "etale_ring_stats": ([P, P, P, P], C.c_int),
            "etale_ring_create": ([P, U32, U32, U32, C.POINTER(P)], C.c_int),
            "etale_ring_buffers": ([P, C.POINTER(P), C.POINTER(U32), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                    C.POINTER(P)], C.c_int),
            "etale_ring_publish": ([P, U64], C.c_int),
            "etale_ring_close": ([P, C.c_int], C.c_int),
            "etale_ring_launch": ([P, U32, U32, C.POINTER(U32), P], C.c_int),
            "etale_ring_destroy": ([P], C.c_int),
            "etale_ring_serve": ([P, P, P, U64, U32, U32, P, P, P, P, C.POINTER(U64), C.POINTER(U32), P], C.c_int),
            "etale_autotune_beam": ([P, P, U64, U32, C.c_float, P, U32, P, C.POINTER(U32), P], C.c_int),
            "etale_export_copies": ([P, U64, U64, P, P, P], C.c_int),
            "etale_set_concurrent": ([P, C.c_int], C.c_int),
            "etale_set_search_tuning": ([P, U32, U32, U32], C.c_int),
            "etale_set_search_keys": ([P, C.c_int], C.c_int),
            "etale_set_exact_rows": ([P, C.c_int], C.c_int),
            "etale_autotune_search": ([P, P, U64, U32, U32, P, U32, C.POINTER(U32), P], C.c_int),
            "etale_search_graph_create": ([P, U32, U32, U32, P, P, P, P, C.POINTER(P)], C.c_int),
            "etale_search_graph_launch": ([P, P], C.c_int),
            "etale_search_graph_check": ([P, P], C.c_int),
            "etale_search_graph_destroy": ([P], C.c_int),
            "etale_selftest_bounded_wait": ([U32, P], C.c_int),
            "etale_ground_truth_info": ([P, P, P], C.c_int),
            "etale_save": ([P, C.c_char_p, P], C.c_int),
            "etale_round_graph_create": ([P, U32, P, U32, P, U32, U32, U32, P, P, P, C.POINTER(P)], C.c_int),
            "etale_round_graph_launch": ([P, P], C.c_int),
            "etale_round_graph_sync": ([P], C.c_int),
            "etale_round_graph_destroy": ([P], C.c_int),
            "etale_search_eval_count": ([P, P, U64, U32, U32, C.POINTER(U64), C.POINTER(U64), C.POINTER(U64), P],
                                        C.c_int),
            "etale_load": ([C.c_char_p, C.POINTER(Config), U64, C.POINTER(P)], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes, f.restype = args, res
        _lib = lib
        return lib


def selftest_bounded_wait(poll_limit: int = 1000, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status code (5 = ETIMEOUT)."""
    return int(load().etale_selftest_bounded_wait(poll_limit, _stream(stream)))


def _ptr(a):
    """Device or host address of a torch tensor or numpy array (contiguous)."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


class Index:
    """One ETALE index on the current CUDA device (see include/etale.h)."""

    def __init__(self, dim: int, metric: str, degree: int, capacity: int, *, build_beam: int = 0,
                 alpha: float = 0.0, max_hops: int = 0, max_cand: int = 0, refine: str = "default",
                 max_batch: int = 0, pool_slabs: int = 0, n_entry: int = 0, mode: str = "deterministic",
                 cas_budget: int = 0, stage_kb: int = 0, gram: str = "default", copies: tuple = (),
                 rerank: int = 0, gt: str = "default", seed: str = "default", exact_rows: str = "off"):
        self.lib = load()
        cfg = Config()
        self.lib.etale_config_default(C.byref(cfg))
        if build_beam:
            cfg.build_beam = build_beam
        if alpha:
            cfg.alpha = alpha
        cfg.max_hops, cfg.max_cand = max_hops, max_cand
        cfg.refine = REFINE[refine]
        cfg.max_batch, cfg.pool_slabs = max_batch, pool_slabs
        if n_entry:
            cfg.n_entry = n_entry
        cfg.mode = MODES[mode]
        if cas_budget:
            cfg.cas_budget = cas_budget
        cfg.stage_kb = stage_kb
        cfg.gram = {"default": 0, "canonical": 1, "tensor": 2}[gram]
        cfg.gt = {"default": 0, "cuda_cores": 1}[gt]
        cfg.seed = {"default": 0, "cuda_cores": 1}[seed]
        cfg.exact_rows = {"off": 0, "on": 1}[exact_rows]
        cfg.copies = (1 if "bf16" in copies else 0) | (2 if "fp8" in copies else 0)
        if rerank:
            cfg.rerank = rerank
        h = C.c_void_p()
        st = self.lib.etale_create(dim, 0 if metric == "l2" else 1, degree, capacity, C.byref(cfg), C.byref(h))
        if st:
            raise EtaleError(st, self.lib.etale_last_error(None).decode())
        self.h = h
        self.dim, self.degree, self.capacity, self.metric = dim, degree, capacity, metric

    def _check(self, st: int):
        if st:
            raise EtaleError(st, self.lib.etale_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.etale_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- snapshots -----------------------------------------------------------
    def save(self, path: str, stream=None):
        """etale_save: write the index state to `path` (format in include/etale.h)."""
        self._check(self.lib.etale_save(self.h, os.fsencode(path), _stream(stream)))

    @classmethod
    def load(cls, path: str, capacity: int = 0) -> "Index":
        """etale_load with the saved configuration; capacity 0 keeps the saved one."""
        lib = load()
        h = C.c_void_p()
        st = lib.etale_load(os.fsencode(path), None, capacity, C.byref(h))
        if st:
            raise EtaleError(st, lib.etale_last_error(None).decode())
        self = cls.__new__(cls)
        self.lib, self.h = lib, h
        s = Stats()
        self._check(lib.etale_stats(h, C.byref(s)))
        self.dim, self.degree, self.capacity = s.dim, s.degree, s.capacity
        self.metric = "l2" if s.metric == 0 else "ip"
        return self

    # --- updates -----------------------------------------------------------
    def insert(self, vecs, stream=None):
        """Insert rows (torch tensor on any device, or numpy); returns the new ids."""
        if not _is_cuda(vecs):
            vecs = np.ascontiguousarray(vecs, dtype=np.float32)
        n = vecs.shape[0]
        ids = np.empty(n, np.uint32)
        self._check(self.lib.etale_insert(self.h, _ptr(vecs), n, _ptr(ids), _stream(stream)))
        return ids

    def delete(self, ids, stream=None) -> int:
        if not _is_cuda(ids):
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
        n = C.c_uint64(0)
        self._check(self.lib.etale_delete(self.h, _ptr(ids), ids.shape[0], C.byref(n), _stream(stream)))
        return int(n.value)

    def reclaim(self, stream=None):
        self._check(self.lib.etale_reclaim(self.h, _stream(stream)))

    # --- queries -----------------------------------------------------------
    def _outputs(self, q, k):
        if _is_cuda(q):
            import torch
            return (torch.empty((q.shape[0], k), dtype=torch.int32, device=q.device),
                    torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device))
        return np.empty((q.shape[0], k), np.uint32), np.empty((q.shape[0], k), np.float32)

    def search(self, queries, k: int, beam: int, stream=None, out=None):
        if not _is_cuda(queries):
            queries = np.ascontiguousarray(queries, dtype=np.float32)
        ids, dist = out if out is not None else self._outputs(queries, k)
        self._check(self.lib.etale_search(self.h, _ptr(queries), queries.shape[0], k, beam, _ptr(ids),
                                          _ptr(dist), _stream(stream)))
        return ids, dist

    def set_exact_rows(self, on: bool = True):
        """Gather the exact BF16 copy in fp32 BeamSearches (see etale_set_exact_rows)."""
        self._check(self.lib.etale_set_exact_rows(self.h, int(on)))

    def set_search_tuning(self, stage_rows: int, seen_bits: int, warps_per_block: int = 0):
        self._check(self.lib.etale_set_search_tuning(self.h, stage_rows, seen_bits, warps_per_block))

    def set_search_keys(self, tensor: bool):
        """BF16 searches: beam keys from the tensor cores (True) or the CUDA cores (False)."""
        self._check(self.lib.etale_set_search_keys(self.h, 1 if tensor else 0))

    def autotune_search(self, queries, k: int, beam: int, stream=None):
        """Time the launch shapes on a device query batch; keep the fastest.
        Returns [(stage_rows, seen_bits, ms, warps_per_block, keys_tc), ...] for the shapes tried."""
        out = (Tuning * 128)()
        n = C.c_uint32(0)
        self._check(self.lib.etale_autotune_search(self.h, _ptr(queries), queries.shape[0], k, beam, out, 128,
                                                   C.byref(n), _stream(stream)))
        return [(out[i].stage_rows, out[i].seen_bits, out[i].ms, out[i].warps_per_block, out[i].keys_tc)
                for i in range(min(n.value, 128))]

    def autotune_beam(self, queries, k: int, target: float, beams=(64, 96, 112, 128, 144, 160, 192, 256),
                      stream=None):
        """etale_autotune_beam: (beam taken, [(beam, recall), ...] tried)."""
        b = np.ascontiguousarray(beams, dtype=np.uint32)
        rec = np.empty(b.size, np.float32)
        ch = C.c_uint32(0)
        self._check(self.lib.etale_autotune_beam(self.h, _ptr(queries), queries.shape[0], k, C.c_float(target),
                                                 _ptr(b), b.size, _ptr(rec), C.byref(ch), _stream(stream)))
        return ch.value, [(int(x), float(r)) for x, r in zip(b, rec) if r >= 0]

    def search_graph(self, queries, out_ids, out_dists, nq_dev, k: int, beam: int) -> "SearchGraph":
        """Capture the query path for batches of up to queries.shape[0] into a CUDA graph."""
        g = C.c_void_p()
        self._check(self.lib.etale_search_graph_create(self.h, queries.shape[0], k, beam, _ptr(queries),
                                                       _ptr(out_ids), _ptr(out_dists), _ptr(nq_dev), C.byref(g)))
        return SearchGraph(self, g)

    def round_graph(self, del_ids, ins_vecs, queries=None, out=None, k: int = 10, beam: int = 64) -> "RoundGraph":
        """Record one churn round over DEVICE tensors: del_ids (int32/uint32, n_del),
        ins_vecs (n_ins x dim), optional queries with out = (ids, dists)."""
        nul = C.c_void_p(None)
        nd = 0 if del_ids is None else del_ids.shape[0]
        ni = 0 if ins_vecs is None else ins_vecs.shape[0]
        nq = 0 if queries is None else queries.shape[0]
        oi, od = out if out is not None else (None, None)
        g = C.c_void_p()
        self._check(self.lib.etale_round_graph_create(
            self.h, nd, _ptr(del_ids) if nd else nul, ni, _ptr(ins_vecs) if ni else nul, nq, k, beam,
            _ptr(queries) if nq else nul, _ptr(oi) if nq else nul, _ptr(od) if nq else nul, C.byref(g)))
        return RoundGraph(self, g, (del_ids, ins_vecs, queries, oi, od))

    def set_concurrent(self, on: bool = True):
        """Let one search thread and one update thread overlap on the device."""
        self._check(self.lib.etale_set_concurrent(self.h, int(on)))

    def set_insert_precision(self, prec: str):
        """"fp32", "bf16" or "fp8" for the BeamSearch of later inserts (rho stays exact fp32)."""
        self._check(self.lib.etale_set_insert_precision(self.h, {"fp32": 0, "bf16": 1, "fp8": 2}[prec]))

    def set_writer_share(self, share: float):
        """Grids of later eager update calls sized for this share of the SMs."""
        self._check(self.lib.etale_set_writer_share(self.h, C.c_float(share)))

    def set_rerank(self, rerank: int):
        """Candidates re-scored in fp32 by reduced-precision queries: rerank * k (at most the beam)."""
        self._check(self.lib.etale_set_rerank(self.h, rerank))

    def set_search_precision(self, prec: str):
        """"fp32", "bf16" or "fp8" for later query searches."""
        self._check(self.lib.etale_set_search_precision(self.h, {"fp32": 0, "bf16": 1, "fp8": 2}[prec]))

    def export_copies(self, first: int, n: int):
        """(bf16 bits uint16[n, dim] or None, fp8 codes uint8[n, dim] or None, scales float32[n] or None)."""
        cfg = self.config()
        b = np.empty((n, self.dim), np.uint16) if cfg["copies"] & 1 else None
        f = np.empty((n, self.dim), np.uint8) if cfg["copies"] & 2 else None
        sc = np.empty(n, np.float32) if cfg["copies"] & 2 else None
        nul = C.c_void_p(None)
        self._check(self.lib.etale_export_copies(self.h, first, n, _ptr(b) if b is not None else nul,
                                                 _ptr(f) if f is not None else nul,
                                                 _ptr(sc) if sc is not None else nul))
        return b, f, sc

    def search_static(self, queries, k: int, beam: int, stream=None, out=None):
        """etale_search_static: device tensors only; allocates nothing on the device."""
        ids, dist = out if out is not None else self._outputs(queries, k)
        self._check(self.lib.etale_search_static(self.h, _ptr(queries), queries.shape[0], k, beam, _ptr(ids),
                                                 _ptr(dist), _stream(stream)))
        return ids, dist

    def eval_count(self, queries, k: int, beam: int, stream=None) -> dict:
        """etale_search_eval_count: evaluations, distinct non-seed ids, expansions."""
        if not _is_cuda(queries):
            queries = np.ascontiguousarray(queries, dtype=np.float32)
        ne, nu, nx = C.c_uint64(), C.c_uint64(), C.c_uint64()
        self._check(self.lib.etale_search_eval_count(self.h, _ptr(queries), queries.shape[0], k, beam, C.byref(ne),
                                                     C.byref(nu), C.byref(nx), _stream(stream)))
        return {"n_eval": ne.value, "n_unique": nu.value, "n_expand": nx.value}

    def ground_truth(self, queries, k: int, stream=None):
        if not _is_cuda(queries):
            queries = np.ascontiguousarray(queries, dtype=np.float32)
        ids, dist = self._outputs(queries, k)
        self._check(self.lib.etale_ground_truth(self.h, _ptr(queries), queries.shape[0], k, _ptr(ids),
                                                _ptr(dist), _stream(stream)))
        return ids, dist

    def ground_truth_info(self) -> dict:
        """How the last ground_truth call ran: path "cuda_cores", "tensor" or
        "tensor_split", and the number of queries recomputed on CUDA cores."""
        path = C.c_uint32()
        fb = C.c_uint64()
        self._check(self.lib.etale_ground_truth_info(self.h, C.byref(path), C.byref(fb)))
        return {"path": ("cuda_cores", "tensor", "tensor_split")[path.value], "fallback_queries": fb.value}

    # --- introspection -----------------------------------------------------
    def export_graph(self, n: int | None = None):
        """(deleted, has_slab, degree, nbr_ids[n, R], nbr_rho[n, R]) over ids [0, n)."""
        n = self.stats()["next_id"] if n is None else n
        R = self.degree
        de, hs, dg = (np.empty(n, np.uint8) for _ in range(3))
        ids = np.empty((n, R), np.uint32)
        rho = np.empty((n, R), np.float32)
        if n:
            self._check(self.lib.etale_export_graph(self.h, n, _ptr(de), _ptr(hs), _ptr(dg), _ptr(ids),
                                                    _ptr(rho), None))
        return de, hs, dg, ids, rho

    def entries(self) -> np.ndarray:
        cap = self.config()["n_entry"]
        out = np.empty(max(cap, 1), np.uint32)
        n = C.c_uint32(0)
        self._check(self.lib.etale_get_entries(self.h, _ptr(out), C.byref(n)))
        return out[:n.value].copy()

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.etale_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def config(self) -> dict:
        c = Config()
        self._check(self.lib.etale_get_config(self.h, C.byref(c)))
        return {f: getattr(c, f) for f, _ in Config._fields_ if f != "reserved"}

    def kernel_launches(self) -> int:
        return int(self.lib.etale_kernel_launches(self.h))

    def set_profiling(self, on: bool = True):
        self._check(self.lib.etale_set_profiling(self.h, int(on)))

    def profile(self, reset: bool = False) -> dict:
        """{phase: (milliseconds, launches)} accumulated while profiling was on."""
        n = len(PHASES)
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.uint64)
        self._check(self.lib.etale_get_profile(self.h, _ptr(ms), _ptr(cnt), n, int(reset)))
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def work(self, reset: bool = False) -> dict:
        """{kind: (row bytes, graph-state bytes)} tallied by the writer kernels."""
        n = len(WORK_KINDS)
        rows = np.zeros(n, np.uint64)
        state = np.zeros(n, np.uint64)
        self._check(self.lib.etale_get_work(self.h, _ptr(rows), _ptr(state), n, int(reset)))
        return {k: (int(rows[i]), int(state[i])) for i, k in enumerate(WORK_KINDS)}


class SearchGraph:
    """A captured query path (see etale_search_graph_create)."""

    def __init__(self, index: Index, handle):
        self.index, self.h = index, handle

    def launch(self, stream=None):
        self.index._check(self.index.lib.etale_search_graph_launch(self.h, _stream(stream)))

    def check(self, stream=None):
        self.index._check(self.index.lib.etale_search_graph_check(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.index.lib.etale_search_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RoundGraph:
    """A recorded churn round (see etale_round_graph_create)."""

    def __init__(self, index: Index, handle, buffers):
        self.index, self.h, self._buffers = index, handle, buffers

    def launch(self, stream=None):
        self.index._check(self.index.lib.etale_round_graph_launch(self.h, _stream(stream)))

    def sync(self):
        self.index._check(self.index.lib.etale_round_graph_sync(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.index.lib.etale_round_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ring:
    """A serving ring (see etale_ring_create): numpy views of the host-mapped
    slots, submission and launches."""

    def __init__(self, index: Index, slots: int, k: int, beam: int):
        self.index, self.slots, self.k = index, slots, k
        h = C.c_void_p()
        index._check(index.lib.etale_ring_create(index.h, slots, k, beam, C.byref(h)))
        self.h = h
        rows, ids, dists, done, served = (C.c_void_p() for _ in range(5))
        stride = C.c_uint32()
        index._check(index.lib.etale_ring_buffers(h, C.byref(rows), C.byref(stride), C.byref(ids), C.byref(dists),
                                                  C.byref(done), C.byref(served)))
        self.stride = stride.value

        def view(p, dtype, shape):
            n = int(np.prod(shape))
            buf = (C.c_byte * (n * np.dtype(dtype).itemsize)).from_address(p.value)
            return np.frombuffer(buf, dtype=dtype).reshape(shape)
        self.rows = view(rows, np.float32, (slots, self.stride))
        self.ids = view(ids, np.uint32, (slots, k))
        self.dists = view(dists, np.float32, (slots, k))
        self.done = view(done, np.uint64, (slots,))
        self.served_by = view(served, np.uint32, (slots,))

    def publish(self, tail: int):
        self.index._check(self.index.lib.etale_ring_publish(self.h, tail))

    def close_ring(self, closed: bool = True):
        self.index._check(self.index.lib.etale_ring_close(self.h, int(closed)))

    def launch(self, max_us: int = 2000, blocks: int = 0, stream=None) -> int:
        seq = C.c_uint32()
        self.index._check(self.index.lib.etale_ring_launch(self.h, max_us, blocks, C.byref(seq), _stream(stream)))
        return seq.value

    def serve(self, queries: np.ndarray, arrival_s: np.ndarray, max_us: int = 2000, blocks: int = 0,
              stream=None) -> dict:
        """etale_ring_serve: queries (host, n x dim) arriving at arrival_s (ascending seconds)."""
        q = np.ascontiguousarray(queries, dtype=np.float32)
        a = np.ascontiguousarray(arrival_s, dtype=np.float64)
        n = q.shape[0]
        issued, done = np.empty(n, np.float64), np.empty(n, np.float64)
        ids, dists = np.empty((n, self.k), np.uint32), np.empty((n, self.k), np.float32)
        mid, nl = C.c_uint64(), C.c_uint32()
        self.index._check(self.index.lib.etale_ring_serve(self.h, _ptr(q), _ptr(a), n, max_us, blocks, _ptr(issued),
                                                          _ptr(done), _ptr(ids), _ptr(dists), C.byref(mid),
                                                          C.byref(nl), _stream(stream)))
        return {"issued": issued, "done": done, "ids": ids, "dists": dists, "mid_launch": mid.value,
                "launches": nl.value}

    def stats(self) -> dict:
        """Queries served and device-clock seconds spent seeding / searching."""
        v = [C.c_uint64(0) for _ in range(3)]
        self.index._check(self.index.lib.etale_ring_stats(self.h, *(C.byref(x) for x in v)))
        return {"served": v[0].value, "seed_s": v[1].value * 1e-9, "search_s": v[2].value * 1e-9}

    def close(self):
        if getattr(self, "h", None):
            self.index.lib.etale_ring_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
