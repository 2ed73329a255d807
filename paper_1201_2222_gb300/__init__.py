"""GB300-native short-characteristics radiative transfer with Jacobi ALI.

The compute path is the CUDA library ``librtsc.so`` (C ABI declared in
``include/rt_sc.h``); :mod:`paper_1201_2222_gb300.rt` is its thin Python
binding.  Importing this package does not load the library; the binding loads
it on first use and raises if it is missing.
"""
__all__ = ["workloads"]
