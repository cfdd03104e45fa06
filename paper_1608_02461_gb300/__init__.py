"""GB300-native FMM-preconditioned GMRES for the 3D Helmholtz equation.

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through ``paper_1608_02461_gb300.hfmm`` (a thin ctypes binding of the
C ABI declared in ``include/hfmm.h``).  Importing this package does not load
the library; ``hfmm.lib()`` does, and raises if it is missing.
"""
