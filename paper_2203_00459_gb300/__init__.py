"""GB300-native decoupled Fourier pose search (Fast-MbyM, arXiv 2203.00459).

The search (Alg. 1) and its adjoint run in the CUDA library libfmbym.so behind the C ABI of
include/fmbym.h; ``search`` is its thin Python face and ``synth`` makes seeded synthetic scans.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "search", "build"]
