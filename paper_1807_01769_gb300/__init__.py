"""GB300-native pseudo-spectral Navier-Stokes hot path (FluidSim, arXiv 1807.01769).

The compute library is ``libns_gb300.so`` (hand-written CUDA for sm_103a behind
a C ABI declared in ``include/ns.h``); ``paper_1807_01769_gb300.ns`` is the thin
ctypes binding.  Importing this package does not load the library.
"""
