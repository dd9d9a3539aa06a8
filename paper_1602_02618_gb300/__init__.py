"""GB300-native (sm_103a) Chebyshev--Jacobi transform.

The compute path is the CUDA library built from ``csrc/`` behind the C ABI of
``include/cjt.h``; ``paper_1602_02618_gb300.cjt`` is the thin ctypes binding.
Importing this package does not load the CUDA library; ``inputs`` holds the
seeded synthetic workload generators.
"""
