"""GB300-native quantics tensor-network Fresnel propagation (arXiv:2510.23089 hot path).

The compute path is the CUDA library ``libqtn.so`` (C ABI in include/qtn.h);
``paper_2510_23089_gb300.qtn`` is its Python binding.  Importing this package
does not load the library; ``qtn.load_library()`` does, and raises if it is
missing.
"""
__all__ = ["qtn", "build"]
