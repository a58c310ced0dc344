"""GB300 (sm_103a) implementation of ETALE's batched dynamic graph ANN maintenance.

The index lives in libetale.so (CUDA, C ABI in include/etale.h); this package
holds its build script, a ctypes binding and the seeded workload generators.
"""
from .binding import Index, EtaleError, load, NIL, EXPORTS, LIB_PATH  # noqa: F401
