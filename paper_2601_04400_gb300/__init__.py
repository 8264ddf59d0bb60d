"""GB300-native FP64 finite-volume Euler/Navier-Stokes step (WENO5 + HLLC + immersed boundary).

The compute path lives in the C-ABI library ``libjaxshock.so`` (``csrc/``); ``binding`` marshals
arguments to it.  Importing this package does not load the library; ``binding.lib()`` does and
raises if it is missing.
"""
__all__ = ["workloads", "binding"]
