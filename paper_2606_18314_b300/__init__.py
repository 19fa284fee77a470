"""B300-native (sm_103a) certificate-maintenance loop for moving points.

Exact nearest-neighbour certificates (nn, d1, d2) for points moving by small
steps in 2-D and 3-D, maintained each step by the validity-radius safety rule,
frontier repair through a uniform-grid index, and the frontier entropy H(F_t)
("Repair Entropy in Dynamic Geometric Nearest-Neighbour Structures", Sec. 2,
Algorithm 1).  The compute runs in hand-written CUDA kernels behind the C ABI
of ``include/cert.h``; ``cert`` is the thin ctypes binding to it.

Importing the package does not load the CUDA library; ``cert`` loads it on
first use and raises if it is missing.
"""
__all__ = ["scenes", "cert"]
