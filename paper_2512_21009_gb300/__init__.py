"""GB300-native dynamic-hypergraph triad-count engine (paper arXiv 2512.21009).

The engine lives in ``libescher.so`` (CUDA for sm_103a, built in-tree by
``build.py``) behind the C ABI of ``include/escher.h``; ``escher`` is its
ctypes binding.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
from . import escher  # noqa: F401
from .escher import (  # noqa: F401
    EscError, Graph, FAMILY_HYPEREDGE, FAMILY_VERTEX, FAMILY_TEMPORAL,
    TRIAD_HYPEREDGE, TRIAD_VERTEX, TRIAD_TEMPORAL,
)
