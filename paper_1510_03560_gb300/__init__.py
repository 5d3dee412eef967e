"""GB300-native progressive-mesh two-component pseudo-potential LBM.

The compute path is the CUDA library ``liblbm`` (C ABI, declared in
``include/lbm.h``); :mod:`paper_1510_03560_gb300.lbm` is its thin ctypes
binding.  Importing the package does not load the library; the first
call into the binding does, and fails loudly when it is missing.
"""

__all__ = ["lbm", "workloads"]
