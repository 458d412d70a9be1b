"""GB300-native finite-volume IMEX update of gray-M1 relativistic radiation MHD
with the PVM-int-8 Jacobian-free Riemann solver (arXiv:2212.00370).

The hot path lives in librrmhd.so (CUDA for sm_103a, C ABI in include/rrmhd.h);
``rrmhd`` is its thin binding, ``workloads`` the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["rrmhd", "workloads", "build"]
