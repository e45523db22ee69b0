"""GB300-native LD-Leiden: device-resident dynamic Leiden updates behind a C ABI.

The package holds the CUDA sources (csrc/), the in-tree build of libldl.so
and the ctypes binding `LDL`.  Importing the package does not load the
library; constructing an LDL does (and fails loudly if it cannot).
"""
from .ldl import LDL, LdlError, Server, apply_batches, load, INSERT, DELETE, REWEIGHT  # noqa: F401
