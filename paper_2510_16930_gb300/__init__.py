"""GB300-native HOQRI hot path (TTMcTC + core update + per-mode QR).

``paper_2510_16930_gb300.hoqri`` binds the CUDA library libhoqri.so
(include/hoqri.h); ``paper_2510_16930_gb300.inputs`` draws the seeded synthetic
workloads.  Importing the package does not load the CUDA library.
"""
