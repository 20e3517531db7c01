"""GB300-native translation-invariant Sinkhorn for entropic unbalanced OT.

The compute path is the CUDA library `libuot.so` (C ABI declared in
include/uot.h); `paper_2201_00730_gb300.uot` binds it.  Importing this package
does not load the library; the first call into `uot` does, and fails loudly
if it is missing.
"""
__all__ = ["uot", "workloads"]
