"""Seeded synthetic inputs shared by the tests, the benchmark, the oracle runs and the GPU runs.

Holds no arithmetic of the method: only the macroscopic initial fields (n, T, u) and seeded random
numbers, with the shapes and value distributions of the paper's workloads (Sec. III) and of the
benchmark cases."""
