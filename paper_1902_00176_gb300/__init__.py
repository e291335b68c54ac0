"""GB300-native Green Function Convolution (GFC) Poisson solver.

The solve runs in the CUDA library built from ``csrc/`` (``libgfc.so``,
C ABI in ``include/gfc.h``); ``paper_1902_00176_gb300.gfc`` is its Python
binding and ``paper_1902_00176_gb300.synth`` the seeded input generators.
"""
