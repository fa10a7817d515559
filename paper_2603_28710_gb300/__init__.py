"""GB300 (sm_103a) asynchronous discontinuous Galerkin operator for compressible Euler.

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/adg.h``);
``adg`` is its thin ctypes binding.  Importing this package does not load the library;
``adg.lib()`` does, and raises if it has not been built.
"""
from . import adg  # noqa: F401
from .adg import AdgError, Solver  # noqa: F401

__all__ = ["adg", "Solver", "AdgError"]
