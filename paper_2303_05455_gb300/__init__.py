"""GB300-native IVHD: the embedding iteration of B. Minch's thesis (arXiv 2303.05455).

The compute path is the CUDA library ``libivhd.so`` (C ABI in ``include/ivhd.h``);
``ivhd`` is its Python binding and ``synth`` the seeded input generators.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "ivhd", "build_lib"]
