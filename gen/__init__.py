"""Seeded synthetic workload generators.

This module is shared by the oracle side and the CUDA side of the tests and
by ``bench.py``.  It only draws random inputs (hyperedge member lists,
timestamps, delete selectors); it holds none of the triad-counting
arithmetic and none of the hyperedge-ID assignment rule, so neither side can
inherit a mistake from the other through it.
"""
from .workloads import *  # noqa: F401,F403
