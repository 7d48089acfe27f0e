"""GB300-native spring-mass simulator (Titan, arXiv 1911.10274, hot path).

The compute path is the C-ABI library ``libtitan.so`` (hand-written sm_103a
kernels behind ``include/titan.h``); ``titan`` is its thin ctypes binding and
``inputs`` builds seeded synthetic systems.  Importing the package loads
nothing; the library is loaded on first use of the binding.
"""
__all__ = ["inputs", "titan"]
