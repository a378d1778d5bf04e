"""GB300 (sm_103a) geodesic landmark shooting with the N-particle Euler-Poincare
system (Camassa, Kuang & Lee, arXiv 1510.03816).

The CUDA library libep.so (C ABI in include/ep.h) holds the whole method; the
``ep`` module is its ctypes binding and ``workloads`` draws seeded synthetic
landmark sets.  Importing the package does not load the library.
"""
__all__ = ["ep", "workloads"]
