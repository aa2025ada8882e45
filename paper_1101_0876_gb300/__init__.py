"""GB300-native checkerboard Metropolis sweep of the 2D q-state Potts model.

The compute path is libpotts.so (hand-written sm_103a CUDA behind a C ABI,
include/potts.h); `potts` is its thin ctypes binding.  Importing this package
does not load the library; `potts.lib()` does, and raises if it is missing.
"""
from . import workloads  # noqa: F401
from .potts import (Batch, Lattice, PottsError, Server,  # noqa: F401
                    threshold_table)
