"""GB300 (sm_103a) engine for exact higher-order U-statistics with graph-factored
kernels (arXiv 2508.12627): U = sum over partitions pi of mu_pi V_pi, every V_pi
an elimination-ordered contraction.

The computation lives in the CUDA library built from csrc/ (libustat.so, C ABI in
include/ustat.h).  ``ustat`` is the ctypes binding, ``engine`` a torch-facing
wrapper, ``build`` the in-tree nvcc build.
"""
__all__ = ["ustat", "engine", "build"]
