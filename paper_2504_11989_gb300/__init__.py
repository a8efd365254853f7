"""GB300 (sm_103a) implementation of the Epstein zeta method for many-body lattice sums.

The compute path is the CUDA library ``_build/libezeta.so`` (C ABI in
``include/ezeta.h``); :mod:`paper_2504_11989_gb300.ezeta` is a thin ctypes binding
with the same names.  Importing the binding raises if the library is missing:
there is no CPU fallback.
"""
from . import workloads  # noqa: F401
