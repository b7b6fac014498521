"""GB300-native ghost-point boundary-condition multigrid (BCMG).

The solver lives in a CUDA shared library (``csrc/``, C ABI declared in
``include/bcmg.h``); ``paper_2207_14208_gb300.bcmg`` is its thin ctypes
binding.  Importing the package does not load the library; the first call
into the binding does, and raises if it is missing.
"""

__all__ = ["bcmg", "workloads"]
