"""B300-native M1 radiative transfer (EMMA, arXiv:1508.07888, Secs. 2.2.3-2.2.4).

The compute path is the C-ABI library ``librt_m1.so`` built from ``csrc/``
(hand-written sm_103a kernels); ``binding`` wraps it with ctypes.  Importing
this package does not load the library: ``binding.lib()`` does, and raises if
the library is missing -- there is no CPU fallback.
"""
__all__ = ["inputs", "binding"]
