"""GB300-native Schwarzschild orbit-library construction and weight solve
(arxiv 2607.00117, "SchwarMAX"): hand-written CUDA for sm_103a behind the
C-ABI in ``include/sw.h``; ``sw`` is its Python binding and ``inputs`` the
seeded synthetic workloads."""
