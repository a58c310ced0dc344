"""Seeded synthetic workloads shaped like the ETALE evaluation (Section 5.2, Table 2).

This module only draws random numbers.  It holds none of the index's
arithmetic and is shared by the CUDA path's tests and bench and by the
oracle's tests, so both sides see the same inputs.

The paper's datasets (SIFT, DEEP, MSONG, Notre, Audio) are replaced by
Gaussian mixtures of matching shape.  Each purpose (mixture centres, base
set, churn inserts, delete choices, queries) draws from its own stream,
spawned from one seed, so changing one part of a workload never shifts the
numbers of another.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

STREAMS = ("centers", "base", "inserts", "deletes", "queries", "assign", "stream", "batches")   # appended only: earlier streams keep their seeds


def _streams(seed: int) -> dict[str, np.random.Generator]:
    ss = np.random.SeedSequence(seed)
    return {name: np.random.Generator(np.random.PCG64(child))
            for name, child in zip(STREAMS, ss.spawn(len(STREAMS)))}


@dataclasses.dataclass(frozen=True)
class Workload:
    """One churn workload: a base set, rounds of deletes + inserts, queries."""
    name: str
    n_base: int
    dim: int
    metric: str            # "l2" or "ip"
    degree: int            # R, the slab capacity
    build_beam: int        # EF_BUILD
    rounds: int
    n_delete: int          # per round
    n_insert: int          # per round
    n_queries: int
    k: int
    search_beam: int       # EF_SEARCH
    n_clusters: int
    kind: str              # generator family, see Mixture
    seed: int = 2607_02543

    @property
    def capacity(self) -> int:
        """Identifier budget: ids are never reused (Proposition 1)."""
        return self.n_base + self.rounds * self.n_insert


# 10,000 x 128 L2 mixture, degree 32, beams 64, 5 rounds of 100 + 100.
SMALL = Workload("gauss64-10k-d128", 10_000, 128, "l2", 32, 64, 5, 100, 100,
                 1_000, 10, 64, 64, "gauss")
# 1,000,000 x 128 integer-valued (0..255) mixture, degree 32, build beam 128,
# 20 rounds of 1% churn (10k deletes + 10k inserts), 10k queries.
SIFT_LIKE_1M = Workload("int256-1m-d128", 1_000_000, 128, "l2", 32, 128, 20,
                        10_000, 10_000, 10_000, 10, 64, 256, "int")


# 1,000,000 x 768 unit vectors (text-embedding shape), inner product, degree 64,
# 1,024 centres, 10 rounds of 1% churn; kept with BF16 and FP8 search copies.
UNIT768_1M = Workload("unit768-1m-ip", 1_000_000, 768, "ip", 64, 128, 10,
                      10_000, 10_000, 10_000, 10, 64, 1024, "unit")
# 1,000,000 x 960 non-negative mixture (512 centres, GIST-like), degree 32;
# 30 rounds of uneven batches (sizes drawn per round, see random_batch_sizes):
# n_delete and n_insert are 0 here, the run draws them.
GIST_LIKE_1M = Workload("absgauss960-1m-d960", 1_000_000, 960, "l2", 32, 128, 30, 0, 0,
                        16_384, 10, 128, 512, "absgauss")
# 10,000,000 x 96 Gaussian mixture (1,000 centres), the served configuration.
GAUSS96_10M = Workload("gauss96-10m-d96", 10_000_000, 96, "l2", 32, 64, 1,
                       0, 0, 1_000, 10, 64, 1000, "gauss")


def scaled(w: Workload, n_base: int, churn_frac: float = 0.01,
           n_queries: int | None = None, rounds: int | None = None) -> Workload:
    """The same mixture family at another size (tests and bounded samples)."""
    n_ch = max(1, int(round(n_base * churn_frac)))
    return dataclasses.replace(
        w, name=f"{w.name}@{n_base}", n_base=n_base, n_delete=n_ch,
        n_insert=n_ch, n_queries=w.n_queries if n_queries is None else n_queries,
        rounds=w.rounds if rounds is None else rounds)


class Mixture:
    """Gaussian mixture generator.

    kind "gauss": centres ~ N(0, 10^2 I), points = centre + N(0, I).
    kind "int":   centres ~ U[0, 255]^m, points = round(centre + 20 N(0, I))
                  clamped to [0, 255] (an integer-valued, SIFT-shaped set).
    kind "unit":  centres uniform on the unit sphere, points =
                  normalise(centre + 0.3 N(0, I/m)).
    kind "absgauss": centres ~ |N(0, 10^2 I)|, points = |centre + N(0, I)|
                  (non-negative, GIST-shaped).
    """

    def __init__(self, w: Workload):
        self.w = w
        self.g = _streams(w.seed)
        m, k = w.dim, w.n_clusters
        gc = self.g["centers"]
        if w.kind == "gauss":
            self.centers = gc.normal(0.0, 10.0, size=(k, m))
        elif w.kind == "absgauss":
            self.centers = np.abs(gc.normal(0.0, 10.0, size=(k, m)))
        elif w.kind == "int":
            self.centers = gc.uniform(0.0, 255.0, size=(k, m))
        elif w.kind == "unit":
            c = gc.normal(size=(k, m))
            self.centers = c / np.linalg.norm(c, axis=1, keepdims=True)
        else:
            raise ValueError(f"unknown mixture kind {w.kind!r}")

    def draw(self, stream: str, n: int, chunk: int = 1 << 16) -> np.ndarray:
        """n fresh points from the mixture on the named stream (float32)."""
        w, g = self.w, self.g[stream]
        out = np.empty((n, w.dim), dtype=np.float32)
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            lab = g.integers(0, w.n_clusters, size=hi - lo)
            noise = g.normal(size=(hi - lo, w.dim))
            c = self.centers[lab]
            if w.kind == "gauss":
                p = c + noise
            elif w.kind == "absgauss":
                p = np.abs(c + noise)
            elif w.kind == "int":
                p = np.clip(np.rint(c + 20.0 * noise), 0.0, 255.0)
            else:
                p = c + (0.3 / math.sqrt(w.dim)) * noise
                p /= np.linalg.norm(p, axis=1, keepdims=True)
            out[lo:hi] = p
        return out


@dataclasses.dataclass
class ChurnPlan:
    base: np.ndarray                 # n_base x dim
    inserts: list[np.ndarray]        # per round, n_insert x dim
    queries: np.ndarray              # n_queries x dim
    delete_rng: np.random.Generator  # draws delete choices round by round


def make_plan(w: Workload) -> ChurnPlan:
    mix = Mixture(w)
    base = mix.draw("base", w.n_base)
    ins_all = mix.draw("inserts", w.rounds * w.n_insert)
    inserts = [ins_all[r * w.n_insert:(r + 1) * w.n_insert] for r in range(w.rounds)]
    queries = mix.draw("queries", w.n_queries)
    return ChurnPlan(base, inserts, queries, mix.g["deletes"])


def choose_deletes(rng: np.random.Generator, live_ids: np.ndarray, n: int) -> np.ndarray:
    """n distinct ids chosen uniformly from the live set (uint32, unsorted)."""
    n = min(n, live_ids.size)
    pick = rng.choice(live_ids.size, size=n, replace=False)
    return live_ids[pick].astype(np.uint32)


def random_batch_sizes(rng: np.random.Generator, n: int, lo: int, hi: int) -> np.ndarray:
    """n sizes drawn log-uniformly in [lo, hi] (uneven batches)."""
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n)).astype(np.int64)
