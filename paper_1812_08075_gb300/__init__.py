"""GB300-native matrix-free SIPG-DG operator (arXiv 1812.08075).

The compute path is the CUDA library libdg (``csrc/``, C ABI in ``include/dg.h``);
``dg`` is its ctypes binding, ``workloads`` the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "dg", "build"]
