"""GB300-native (sm_103a) exponential integrators for complex Ginzburg-Landau
equations (Caliari & Cassini, arXiv 2403.02816).

The compute path is the C-ABI library ``lib/libcgl.so`` (hand-written CUDA);
``native`` is its thin ctypes binding.  ``inputs`` holds the seeded synthetic
workloads.  Importing the package does not load the library.
"""
__all__ = ["inputs", "native"]
