"""GB300-native ε-distance similarity self-join (arXiv 1809.09930 method).

The compute path is the CUDA library ``libgj.so`` (sources in ``csrc/``, C ABI
in ``include/gj.h``); ``gj`` is its Python binding.
"""
from . import gj  # noqa: F401
from .gj import Index  # noqa: F401

__all__ = ["gj", "Index"]
