"""ctypes front-end of the C oracle (``escher_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline of the benchmark.  The product path never imports this module.

Families are selected with the same bit values the public header documents
(1 hyperedge, 2 incident-vertex, 4 temporal); the oracle restates them here
on purpose rather than importing the product's constants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

from .rebuild import OracleHypergraph

FAM_HYPEREDGE = 1
FAM_VERTEX = 2
FAM_TEMPORAL = 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "escher_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_ERRORS = {1: "bad input", 2: "count overflows uint64", 3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               _SRC, "-o", _LIB])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        p64, p32, pu64 = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_uint64)
        for name in ("orc_num_static_classes", "orc_num_static_classes_nodup",
                     "orc_num_temporal_classes"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = []
        for name in ("orc_static_rep", "orc_static_closed", "orc_static_dup",
                     "orc_static_class_of_mask", "orc_temporal_class_of_mask",
                     "orc_temporal_mask"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_int]
        for name in ("orc_count_brute", "orc_count_wedge"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_int64, p64, p32, p64, p32, C.c_int64, C.c_uint32, pu64, pu64]
        L.orc_count_containing.restype = C.c_int
        L.orc_count_containing.argtypes = [C.c_int64, p64, p32, p64, p32, C.c_int64, C.c_uint32,
                                           C.c_int64, p64, pu64, pu64]
        L.orc_vertex_literal.restype = C.c_int
        L.orc_vertex_literal.argtypes = [C.c_int64, p64, p32, C.c_int32, pu64]
        L.orc_vertex_triples.restype = C.c_int
        L.orc_vertex_triples.argtypes = [C.c_int64, p64, p32, pu64]
        L.orc_vertex_literal_containing.restype = C.c_int
        L.orc_vertex_literal_containing.argtypes = [C.c_int64, p64, p32, C.c_int32, C.POINTER(C.c_uint8), pu64]
        L.orc_vertex_containing.restype = C.c_int
        L.orc_vertex_containing.argtypes = [C.c_int64, p64, p32, C.c_int64, p64, pu64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}: {_ERRORS.get(rc, '?')}")


# ---------------------------------------------------------------------------
# class tables
# ---------------------------------------------------------------------------

def tables() -> dict:
    L = lib()
    ns, nt = L.orc_num_static_classes(), L.orc_num_temporal_classes()
    return dict(
        n_static=ns,
        n_static_nodup=L.orc_num_static_classes_nodup(),
        n_temporal=nt,
        static_rep=[L.orc_static_rep(i) for i in range(ns)],
        static_closed=[L.orc_static_closed(i) for i in range(ns)],
        static_dup=[L.orc_static_dup(i) for i in range(ns)],
        static_of_mask=[L.orc_static_class_of_mask(m) for m in range(128)],
        temporal_of_mask=[L.orc_temporal_class_of_mask(m) for m in range(128)],
        temporal_mask=[L.orc_temporal_mask(i) for i in range(nt)],
    )


# ---------------------------------------------------------------------------
# counting on a CSR of live hyperedges (members sorted, unique)
# ---------------------------------------------------------------------------

def _prep(off, mem, ts, ids):
    off = np.ascontiguousarray(off, dtype=np.int64)
    mem = np.ascontiguousarray(mem, dtype=np.int32)
    n = off.shape[0] - 1
    ts = np.ascontiguousarray(np.zeros(n, np.int64) if ts is None else ts, dtype=np.int64)
    ids = np.ascontiguousarray(np.arange(n, dtype=np.int32) if ids is None else ids, dtype=np.int32)
    if mem.size == 0:
        mem = np.zeros(1, np.int32)
    return n, off, mem, ts, ids


def count_hyperedge_temporal(off, mem, ts=None, ids=None, delta: int = 0,
                             families: int = FAM_HYPEREDGE | FAM_TEMPORAL,
                             method: str = "wedge"):
    """(h30, t96) uint64 arrays over the given live hyperedges."""
    n, off, mem, ts, ids = _prep(off, mem, ts, ids)
    h30 = np.zeros(30, np.uint64)
    t96 = np.zeros(96, np.uint64)
    fn = {"brute": lib().orc_count_brute, "wedge": lib().orc_count_wedge}[method]
    _check(fn(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32), _ptr(ts, C.c_int64),
              _ptr(ids, C.c_int32), int(delta), int(families),
              _ptr(h30, C.c_uint64), _ptr(t96, C.c_uint64)))
    return h30, t96


def count_containing(off, mem, ts, ids, delta: int, families: int, sel_pos: Sequence[int]):
    """(h30, t96) over the connected triples containing >= 1 of the hyperedges
    at the given positions of the CSR."""
    n, off, mem, ts, ids = _prep(off, mem, ts, ids)
    sel = np.ascontiguousarray(sel_pos, dtype=np.int64)
    h30 = np.zeros(30, np.uint64)
    t96 = np.zeros(96, np.uint64)
    _check(lib().orc_count_containing(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32),
                                      _ptr(ts, C.c_int64), _ptr(ids, C.c_int32), int(delta),
                                      int(families), sel.size, _ptr(sel, C.c_int64),
                                      _ptr(h30, C.c_uint64), _ptr(t96, C.c_uint64)))
    return h30, t96


def count_vertex(off, mem, n_vertices: Optional[int] = None, method: str = "triples"):
    """uint64[3]: incident-vertex triads of types 1, 2, 3."""
    n, off, mem, _, _ = _prep(off, mem, None, None)
    v3 = np.zeros(3, np.uint64)
    if method == "literal":
        _check(lib().orc_vertex_literal(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32),
                                        int(n_vertices), _ptr(v3, C.c_uint64)))
    else:
        _check(lib().orc_vertex_triples(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32),
                                        _ptr(v3, C.c_uint64)))
    return v3


def count_vertex_containing(off, mem, sel_pos: Sequence[int], n_vertices: Optional[int] = None,
                            method: str = "triples"):
    """uint64[3]: incident-vertex instances (types 1, 2, 3) with at least one
    witness among the hyperedges at the given positions of the CSR."""
    n, off, mem, _, _ = _prep(off, mem, None, None)
    v3 = np.zeros(3, np.uint64)
    if method == "literal":
        sel = np.zeros(max(n, 1), np.uint8)
        sel[np.asarray(sel_pos, dtype=np.int64)] = 1
        _check(lib().orc_vertex_literal_containing(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32),
                                                   int(n_vertices), _ptr(sel, C.c_uint8),
                                                   _ptr(v3, C.c_uint64)))
    else:
        sp = np.ascontiguousarray(sel_pos, dtype=np.int64)
        _check(lib().orc_vertex_containing(n, _ptr(off, C.c_int64), _ptr(mem, C.c_int32), sp.size,
                                           _ptr(sp, C.c_int64), _ptr(v3, C.c_uint64)))
    return v3


def counts(g: OracleHypergraph, families: int, delta: int = 0, method: str = "wedge") -> dict:
    """All requested families of the live hypergraph ``g``, recounted from
    scratch: {"hyperedge": u64[30], "vertex": u64[3], "temporal": u64[96]}."""
    off, mem, ts, ids = g.csr()
    out = {}
    if families & (FAM_HYPEREDGE | FAM_TEMPORAL):
        h30, t96 = count_hyperedge_temporal(off, mem, ts, ids, delta, families, method)
        if families & FAM_HYPEREDGE:
            out["hyperedge"] = h30
        if families & FAM_TEMPORAL:
            out["temporal"] = t96
    if families & FAM_VERTEX:
        out["vertex"] = count_vertex(off, mem, g.n_vertices,
                                     "literal" if method == "literal" else "triples")
    return out
