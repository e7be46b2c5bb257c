"""GB300-native preconditioned discrete dipole approximation (arXiv 1903.09802).

The computation lives in ``libdda.so`` (CUDA, sm_103a) behind the C ABI of
``include/dda.h``; ``paper_1903_09802_gb300.dda`` is its Python binding.
Build the library with ``paper_1903_09802_gb300.build.build()``.
"""
from .build import LIB, build  # noqa: F401

__all__ = ["build", "LIB"]
