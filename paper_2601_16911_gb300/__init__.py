"""GB300 (sm_103a) cell-vertex WENO stabilised DG solver.

The compute path lives in the CUDA library ``_build/libcvweno.so`` (sources in
``csrc/``, ABI in ``include/cvweno.h``); ``cvweno`` is its thin ctypes binding and
``inputs`` the seeded synthetic workloads.  Importing the package does not load the
library; ``cvweno.load()`` does, and fails loudly when it has not been built.
"""
__all__ = ["cvweno", "inputs", "build"]
