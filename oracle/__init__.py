"""ETALE oracle: the sequential CPU restatement in etale_oracle.c and its loader.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs import this package.  The product path never
does, and the oracle shares no source with it.
"""
from .oracle import Oracle, build, dist, dist64, robust_prune_vectors, NIL  # noqa: F401
