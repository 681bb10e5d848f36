"""Python binding of the C ABI in include/escher.h (ctypes).

Argument marshalling only: the functions named like the C entry points
(``esc_create``, ``esc_apply_batch``, ``esc_triads``, ``esc_destroy``, ...)
turn numpy arrays or torch tensors into pointers and call the library; all
work happens in the CUDA kernels behind the ABI.  There is no fallback: if
``libescher.so`` has not been built, importing the library raises.

Arrays may live on the host (numpy, CPU tensors) or on the device (CUDA
tensors); the library tells them apart.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libescher.so")

FAMILY_HYPEREDGE = 1
FAMILY_VERTEX = 2
FAMILY_TEMPORAL = 4
FAMILY_VERTEX12 = 8
TRIAD_HYPEREDGE, TRIAD_VERTEX, TRIAD_TEMPORAL = 0, 1, 2
N_CLASSES = {TRIAD_HYPEREDGE: 30, TRIAD_VERTEX: 3, TRIAD_TEMPORAL: 96}
STATUS = {0: "ESC_OK", 1: "ESC_ERR_INVALID_ARG", 2: "ESC_ERR_NOT_FOUND", 3: "ESC_ERR_OUT_OF_MEMORY",
          4: "ESC_ERR_UNSUPPORTED", 5: "ESC_ERR_TIMEOUT", 6: "ESC_ERR_CUDA", 7: "ESC_ERR_BUSY",
          8: "ESC_ERR_INTERNAL"}
ESC_ERR_BUSY = 7

# every symbol the header declares (checked by the CPU test suite)
EXPORTED = [
    "esc_create", "esc_apply_batch", "esc_triads", "esc_local_triads", "esc_destroy", "esc_last_error",
    "esc_export_sizes", "esc_export", "esc_set_profiling", "esc_last_stats", "esc_launch_count",
    "esc_group_create", "esc_group_apply", "esc_group_triads", "esc_group_destroy",
    "esc_group_last_error", "esc_group_set_profiling", "esc_group_last_stats", "esc_group_launch_count",
    "esc_group_bytes", "esc_server_create", "esc_server_submit", "esc_server_wait", "esc_server_drain",
    "esc_server_triads", "esc_server_get_stats", "esc_server_destroy", "esc_autotune", "esc_group_autotune",
    "esc_set_graph_launch", "esc_group_set_graph_launch", "esc_update_members", "esc_group_update_members",
    "esc_version", "esc_count_static_noalloc", "esc_insert_with_ids", "esc_restore",
    "esc_group_insert_with_ids", "esc_group_export_sizes", "esc_group_export", "esc_export_h2h",
    "esc_group_export_h2h", "esc_set_split", "esc_group_set_split", "esc_server_add_group", "esc_group_fits",
]


class EscError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class esc_config(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("capacity_hyperedges", C.c_int64),
                ("capacity_incidences", C.c_int64), ("max_batch_hyperedges", C.c_int64),
                ("max_batch_incidences", C.c_int64), ("families", C.c_uint32), ("delta", C.c_int64),
                ("debug", C.c_int32), ("capacity_vertex_pairs", C.c_int64)]


class esc_batch_stats(C.Structure):
    _fields_ = [("ms_total", C.c_float), ("ms_ingest", C.c_float), ("ms_count_del", C.c_float),
                ("ms_store", C.c_float), ("ms_count_ins", C.c_float), ("launches", C.c_int64),
                ("count_launches", C.c_int64), ("v2h_reads", C.c_int64), ("h2v_reads", C.c_int64),
                ("meta_reads", C.c_int64), ("triads", C.c_int64), ("alg_entries", C.c_int64),
                ("work", C.c_int64 * 6), ("ms_center", C.c_float), ("center_launches", C.c_int32),
                ("alg_center", C.c_int64), ("alg_store", C.c_int64), ("alg_build", C.c_int64),
                ("alg_closed", C.c_int64), ("alg_open", C.c_int64)]


class esc_batch(C.Structure):
    _fields_ = [("graph", C.c_int32), ("n_ins", C.c_int64), ("ins_offsets", C.c_void_p),
                ("ins_members", C.c_void_p), ("ins_timestamps", C.c_void_p), ("n_del", C.c_int64),
                ("del_ids", C.c_void_p), ("out_ins_ids", C.c_void_p)]


class esc_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("call_batches", C.c_int32), ("t_arrival_ns", C.c_int64),
                ("t_start_ns", C.c_int64), ("t_done_ns", C.c_int64), ("call_updates", C.c_int64)]


class esc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("rejected", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("calls", C.c_int64), ("updates", C.c_int64),
                ("pending_updates", C.c_int64)]


class esc_tune_result(C.Structure):
    _fields_ = [("center_shape", C.c_int32), ("restricted", C.c_int32), ("ms", C.c_float * 8),
                ("table_from", C.c_int32), ("m1_pct", C.c_int32), ("ms_table", C.c_float * 3),
                ("ms_m1", C.c_float * 3)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    st = C.c_int
    L.esc_create.argtypes = [C.POINTER(esc_config), i64, vp, vp, vp, vp, C.POINTER(vp)]
    L.esc_apply_batch.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp]
    L.esc_triads.argtypes = [vp, C.c_int, i64, vp, i32]
    L.esc_local_triads.argtypes = [vp, i64, vp, vp, vp, vp]
    L.esc_destroy.argtypes = [vp]
    L.esc_last_error.argtypes = [vp]
    L.esc_last_error.restype = C.c_char_p
    L.esc_export_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.esc_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.esc_set_profiling.argtypes = [vp, i32]
    L.esc_last_stats.argtypes = [vp, C.POINTER(esc_batch_stats)]
    L.esc_launch_count.argtypes = [vp]
    L.esc_launch_count.restype = i64
    L.esc_group_create.argtypes = [C.POINTER(esc_config), i32, C.POINTER(esc_config), vp, C.POINTER(vp)]
    L.esc_group_apply.argtypes = [vp, i32, C.POINTER(esc_batch)]
    L.esc_group_triads.argtypes = [vp, i32, C.c_int, i64, vp, i32]
    L.esc_group_destroy.argtypes = [vp]
    L.esc_group_last_error.argtypes = [vp]
    L.esc_group_last_error.restype = C.c_char_p
    L.esc_group_set_profiling.argtypes = [vp, i32]
    L.esc_group_last_stats.argtypes = [vp, C.POINTER(esc_batch_stats)]
    L.esc_group_launch_count.argtypes = [vp]
    L.esc_group_launch_count.restype = i64
    L.esc_group_bytes.argtypes = [C.POINTER(esc_config), i32, C.POINTER(esc_config), C.POINTER(i64)]
    L.esc_server_create.argtypes = [vp, i64, i32, C.POINTER(vp)]
    L.esc_server_submit.argtypes = [vp, C.POINTER(esc_batch), i64, C.POINTER(i64)]
    L.esc_server_wait.argtypes = [vp, i64, C.POINTER(esc_request_info)]
    L.esc_server_drain.argtypes = [vp]
    L.esc_server_triads.argtypes = [vp, i32, C.c_int, i64, vp, i32]
    L.esc_server_get_stats.argtypes = [vp, C.POINTER(esc_server_stats)]
    L.esc_server_destroy.argtypes = [vp]
    L.esc_autotune.argtypes = [vp, i64, vp, i32, C.POINTER(esc_tune_result)]
    L.esc_set_graph_launch.argtypes = [vp, i32]
    L.esc_set_split.argtypes = [vp, i32, i32]
    L.esc_server_add_group.argtypes = [vp, vp, C.POINTER(i32)]
    L.esc_group_fits.argtypes = [C.POINTER(esc_config), i32, C.POINTER(esc_config), i64, C.POINTER(i32)]
    L.esc_group_set_split.argtypes = [vp, i32, i32]
    L.esc_update_members.argtypes = [vp, i64, vp, vp, vp]
    L.esc_group_update_members.argtypes = [vp, i32, i64, vp, vp, vp]
    L.esc_group_set_graph_launch.argtypes = [vp, i32]
    L.esc_group_autotune.argtypes = [vp, i32, i64, vp, i32, C.POINTER(esc_tune_result)]
    L.esc_insert_with_ids.argtypes = [vp, i64, vp, vp, vp, vp]
    L.esc_restore.argtypes = [C.POINTER(esc_config), i64, vp, vp, vp, vp, vp, C.POINTER(vp)]
    L.esc_group_insert_with_ids.argtypes = [vp, i32, i64, vp, vp, vp, vp]
    L.esc_group_export_sizes.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i64)]
    L.esc_group_export.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
    L.esc_export_h2h.argtypes = [vp, i32, C.POINTER(i64), vp, vp, vp]
    L.esc_group_export_h2h.argtypes = [vp, i32, i32, C.POINTER(i64), vp, vp, vp]
    L.esc_version.restype = C.c_char_p
    L.esc_count_static_noalloc.argtypes = [i32, i64, vp, vp, vp, u32, i64, vp, vp]
    L.esc_count_static_noalloc.restype = st
    for name in ("esc_create", "esc_apply_batch", "esc_triads", "esc_local_triads", "esc_destroy",
                 "esc_export_sizes", "esc_export", "esc_set_profiling", "esc_last_stats",
                 "esc_group_create", "esc_group_apply", "esc_group_triads", "esc_group_destroy",
                 "esc_group_set_profiling", "esc_group_last_stats", "esc_group_bytes", "esc_server_create",
                 "esc_server_submit", "esc_server_wait", "esc_server_drain", "esc_server_triads",
                 "esc_server_get_stats", "esc_server_destroy", "esc_autotune", "esc_group_autotune",
                 "esc_set_graph_launch", "esc_group_set_graph_launch", "esc_update_members",
                 "esc_group_update_members", "esc_insert_with_ids", "esc_restore", "esc_group_insert_with_ids",
                 "esc_group_export_sizes", "esc_group_export", "esc_export_h2h", "esc_group_export_h2h",
                 "esc_set_split", "esc_group_set_split", "esc_server_add_group", "esc_group_fits"):
        getattr(L, name).restype = st
    _lib = L
    return L


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------

def _ptr(a, dtype):
    """Pointer of a numpy array or torch tensor (converted to ``dtype`` and
    made contiguous when needed); returns (pointer, keep-alive object)."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.int64}[dtype]
            t = a.to(tdt).contiguous()
            return (t.data_ptr() if t.numel() else None), t
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return (arr.ctypes.data if arr.size else None), arr


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(rc, err_fn, handle):
    if rc != 0:
        msg = err_fn(handle)
        raise EscError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# same names as the C ABI
# ---------------------------------------------------------------------------

def esc_create(cfg: esc_config, offsets, members, timestamps=None, stream=None) -> int:
    L = load()
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    pt, kt = _ptr(timestamps, np.int64)
    n_he = (len(offsets) - 1) if offsets is not None else 0
    h = C.c_void_p()
    rc = L.esc_create(C.byref(cfg), n_he, po, pm, pt, _stream_ptr(stream), C.byref(h))
    _check(rc, L.esc_last_error, None)
    return h.value


def esc_apply_batch(g: int, ins_offsets, ins_members, ins_timestamps, del_ids, out_ids=None) -> None:
    L = load()
    po, ko = _ptr(ins_offsets, np.int64)
    pm, km = _ptr(ins_members, np.int32)
    pt, kt = _ptr(ins_timestamps, np.int64)
    pd, kd = _ptr(del_ids, np.int32)
    n_ins = (len(ins_offsets) - 1) if ins_offsets is not None and len(ins_offsets) else 0
    n_del = len(del_ids) if del_ids is not None else 0
    pout = None
    if out_ids is not None:
        pout = out_ids.ctypes.data if isinstance(out_ids, np.ndarray) else out_ids.data_ptr()
    rc = L.esc_apply_batch(g, n_ins, po, pm, pt, n_del, pd, pout)
    _check(rc, L.esc_last_error, g)


def esc_triads(g: int, triad_type: int, window: int = 0) -> np.ndarray:
    L = load()
    n = N_CLASSES[triad_type]
    out = np.zeros(n, np.uint64)
    rc = L.esc_triads(g, triad_type, window, out.ctypes.data, n)
    _check(rc, L.esc_last_error, g)
    return out


def esc_local_triads(g: int, ids):
    L = load()
    pi, ki = _ptr(ids, np.int32)
    oh, ov, ot = np.zeros(30, np.uint64), np.zeros(3, np.uint64), np.zeros(96, np.uint64)
    rc = L.esc_local_triads(g, len(ids), pi, oh.ctypes.data, ov.ctypes.data, ot.ctypes.data)
    _check(rc, L.esc_last_error, g)
    return oh, ov, ot


def esc_destroy(g: int) -> None:
    if g:
        load().esc_destroy(g)


def _export_arrays(n: int, m: int, n_vertices: int):
    return (np.zeros(max(n, 1), np.int32), np.zeros(max(n, 1), np.int64), np.zeros(n + 1, np.int64),
            np.zeros(max(m, 1), np.int32), np.zeros(n_vertices + 1, np.int64), np.zeros(max(m, 1), np.int32))


def esc_group_export(grp: int, graph: int, n_vertices: int) -> dict:
    """Graph ``graph`` of the group as esc_export gives it (its own IDs)."""
    L = load()
    nl, ni = C.c_int64(), C.c_int64()
    _check(L.esc_group_export_sizes(grp, int(graph), C.byref(nl), C.byref(ni)), L.esc_group_last_error, grp)
    n, m = nl.value, ni.value
    ids, ts, off, mem, voff, vmem = _export_arrays(n, m, n_vertices)
    rc = L.esc_group_export(grp, int(graph), ids.ctypes.data, ts.ctypes.data, off.ctypes.data, mem.ctypes.data,
                            voff.ctypes.data, vmem.ctypes.data)
    _check(rc, L.esc_group_last_error, grp)
    return dict(ids=ids[:n], timestamps=ts[:n], offsets=off, members=mem[:m], v_offsets=voff,
                v_members=vmem[:m])


def _h2h(call, err, handle, n_live: int, s: int) -> dict:
    n = C.c_int64()
    off = np.zeros(n_live + 1, np.int64)
    _check(call(C.byref(n), off.ctypes.data, None, None), err, handle)
    nbr = np.zeros(max(n.value, 1), np.int32)
    ov = np.zeros(max(n.value, 1), np.int32)
    _check(call(C.byref(n), off.ctypes.data, nbr.ctypes.data, ov.ctypes.data), err, handle)
    return dict(offsets=off, neighbours=nbr[:n.value], overlaps=ov[:n.value])


def esc_export_h2h(g: int, s: int = 1) -> dict:
    """Line graph (s = 1) or s-line graph: per live hyperedge, in ascending
    ID order, the hyperedges sharing at least s vertices and how many."""
    L = load()
    nl = C.c_int64()
    _check(L.esc_export_sizes(g, C.byref(nl), None), L.esc_last_error, g)
    return _h2h(lambda *a: L.esc_export_h2h(g, int(s), *a), L.esc_last_error, g, nl.value, s)


def esc_group_export_h2h(grp: int, graph: int, s: int = 1) -> dict:
    L = load()
    nl = C.c_int64()
    _check(L.esc_group_export_sizes(grp, int(graph), C.byref(nl), None), L.esc_group_last_error, grp)
    return _h2h(lambda *a: L.esc_group_export_h2h(grp, int(graph), int(s), *a), L.esc_group_last_error, grp,
                nl.value, s)


def esc_insert_with_ids(g: int, ids, offsets, members, timestamps=None) -> None:
    """Insert hyperedge j under ID ids[j] (a free ID)."""
    L = load()
    pi, ki = _ptr(ids, np.int32)
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    pt, kt = _ptr(timestamps, np.int64)
    _check(L.esc_insert_with_ids(g, len(ids), pi, po, pm, pt), L.esc_last_error, g)


def esc_group_insert_with_ids(grp: int, graph: int, ids, offsets, members, timestamps=None) -> None:
    L = load()
    pi, ki = _ptr(ids, np.int32)
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    pt, kt = _ptr(timestamps, np.int64)
    _check(L.esc_group_insert_with_ids(grp, int(graph), len(ids), pi, po, pm, pt), L.esc_group_last_error, grp)


def esc_restore(cfg: esc_config, ids, offsets, members, timestamps=None, stream=None) -> int:
    """A new graph holding the hyperedges of an export, under their IDs."""
    L = load()
    pi, ki = _ptr(ids, np.int32)
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    pt, kt = _ptr(timestamps, np.int64)
    h = C.c_void_p()
    rc = L.esc_restore(C.byref(cfg), len(ids), pi, po, pm, pt, _stream_ptr(stream), C.byref(h))
    _check(rc, L.esc_last_error, None)
    return h.value


def esc_export(g: int, n_vertices: int) -> dict:
    L = load()
    nl, ni = C.c_int64(), C.c_int64()
    _check(L.esc_export_sizes(g, C.byref(nl), C.byref(ni)), L.esc_last_error, g)
    n, m = nl.value, ni.value
    ids, ts, off, mem, voff, vmem = _export_arrays(n, m, n_vertices)
    rc = L.esc_export(g, ids.ctypes.data, ts.ctypes.data, off.ctypes.data, mem.ctypes.data,
                      voff.ctypes.data, vmem.ctypes.data)
    _check(rc, L.esc_last_error, g)
    return dict(ids=ids[:n], timestamps=ts[:n], offsets=off, members=mem[:m], v_offsets=voff,
                v_members=vmem[:m])


def esc_last_stats(g: int) -> dict:
    L = load()
    s = esc_batch_stats()
    _check(L.esc_last_stats(g, C.byref(s)), L.esc_last_error, g)
    return {k: (list(getattr(s, k)) if k == "work" else getattr(s, k)) for k, _ in esc_batch_stats._fields_}


def esc_set_profiling(g: int, on: bool) -> None:
    load().esc_set_profiling(g, 1 if on else 0)


def esc_launch_count(g: int) -> int:
    return int(load().esc_launch_count(g))


def esc_version() -> str:
    return load().esc_version().decode()


def esc_group_create(shared: esc_config, graph_cfgs: Sequence[esc_config], stream=None) -> int:
    L = load()
    arr = (esc_config * len(graph_cfgs))(*graph_cfgs)
    h = C.c_void_p()
    rc = L.esc_group_create(C.byref(shared), len(graph_cfgs), arr, _stream_ptr(stream), C.byref(h))
    _check(rc, L.esc_group_last_error, None)
    return h.value


def esc_group_bytes(shared: esc_config, graph_cfgs: Sequence[esc_config]) -> int:
    """Device bytes esc_group_create would allocate (nothing is allocated)."""
    L = load()
    arr = (esc_config * len(graph_cfgs))(*graph_cfgs)
    out = C.c_int64(0)
    rc = L.esc_group_bytes(C.byref(shared), len(graph_cfgs), arr, C.byref(out))
    if rc != 0:
        raise EscError(rc, "esc_group_bytes failed")
    return int(out.value)


def esc_group_apply(grp: int, batches: Sequence[dict]) -> None:
    """batches: dicts with graph, ins_offsets, ins_members, ins_timestamps,
    del_ids and optionally out_ids (a writable int32 numpy array)."""
    L = load()
    keep = []
    arr = (esc_batch * len(batches))()
    for i, b in enumerate(batches):
        po, ko = _ptr(b.get("ins_offsets"), np.int64)
        pm, km = _ptr(b.get("ins_members"), np.int32)
        pt, kt = _ptr(b.get("ins_timestamps"), np.int64)
        pd, kd = _ptr(b.get("del_ids"), np.int32)
        keep += [ko, km, kt, kd]
        off = b.get("ins_offsets")
        dl = b.get("del_ids")
        out = b.get("out_ids")
        arr[i].graph = int(b["graph"])
        arr[i].n_ins = (len(off) - 1) if off is not None and len(off) else 0
        arr[i].ins_offsets = po
        arr[i].ins_members = pm
        arr[i].ins_timestamps = pt
        arr[i].n_del = len(dl) if dl is not None else 0
        arr[i].del_ids = pd
        arr[i].out_ins_ids = (out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()) \
            if out is not None else None
    rc = L.esc_group_apply(grp, len(batches), arr)
    _check(rc, L.esc_group_last_error, grp)


def esc_group_triads(grp: int, graph: int, triad_type: int, window: int = 0) -> np.ndarray:
    L = load()
    n = N_CLASSES[triad_type]
    out = np.zeros(n, np.uint64)
    rc = L.esc_group_triads(grp, graph, triad_type, window, out.ctypes.data, n)
    _check(rc, L.esc_group_last_error, grp)
    return out


def esc_group_destroy(grp: int) -> None:
    if grp:
        load().esc_group_destroy(grp)


def esc_group_set_profiling(grp: int, on: bool) -> None:
    load().esc_group_set_profiling(grp, 1 if on else 0)


def esc_group_last_stats(grp: int) -> dict:
    L = load()
    s = esc_batch_stats()
    _check(L.esc_group_last_stats(grp, C.byref(s)), L.esc_group_last_error, grp)
    return {k: (list(getattr(s, k)) if k == "work" else getattr(s, k)) for k, _ in esc_batch_stats._fields_}


def esc_group_launch_count(grp: int) -> int:
    return int(load().esc_group_launch_count(grp))


def _tune_dict(r: "esc_tune_result") -> dict:
    return {"center_shape": r.center_shape, "restricted": r.restricted, "ms": list(r.ms),
            "table_from": r.table_from, "m1_pct": r.m1_pct, "ms_table": list(r.ms_table), "ms_m1": list(r.ms_m1)}


def esc_autotune(h: int, ids, reps: int = 2) -> dict:
    """Time the counter's launch shapes on the triads of the live hyperedges
    ``ids`` and keep the fastest; returns the choice and every timing."""
    L = load()
    p, keep = _ptr(ids, np.int32)
    r = esc_tune_result()
    rc = L.esc_autotune(h, len(ids), p, int(reps), C.byref(r))
    _check(rc, L.esc_last_error, h)
    return _tune_dict(r)


def esc_update_members(h: int, ids, offsets, members) -> None:
    """Horizontal update: live hyperedge ids[j] gets the vertex set
    members[offsets[j]:offsets[j+1]] and keeps its ID and timestamp."""
    L = load()
    pi, ki = _ptr(ids, np.int32)
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    _check(L.esc_update_members(h, len(ids), pi, po, pm), L.esc_last_error, h)


def esc_group_update_members(grp: int, graph: int, ids, offsets, members) -> None:
    L = load()
    pi, ki = _ptr(ids, np.int32)
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    _check(L.esc_group_update_members(grp, int(graph), len(ids), pi, po, pm), L.esc_group_last_error, grp)


def esc_set_graph_launch(h: int, on: bool = True) -> None:
    L = load()
    _check(L.esc_set_graph_launch(h, 1 if on else 0), L.esc_last_error, h)


def esc_group_set_graph_launch(grp: int, on: bool = True) -> None:
    L = load()
    _check(L.esc_group_set_graph_launch(grp, 1 if on else 0), L.esc_group_last_error, grp)


def esc_set_split(h: int, rank: int, world: int) -> None:
    L = load()
    _check(L.esc_set_split(h, int(rank), int(world)), L.esc_last_error, h)


def esc_group_set_split(grp: int, rank: int, world: int) -> None:
    L = load()
    _check(L.esc_group_set_split(grp, int(rank), int(world)), L.esc_group_last_error, grp)


def esc_group_autotune(grp: int, graph: int, ids, reps: int = 2) -> dict:
    L = load()
    p, keep = _ptr(ids, np.int32)
    r = esc_tune_result()
    rc = L.esc_group_autotune(grp, int(graph), len(ids), p, int(reps), C.byref(r))
    _check(rc, L.esc_group_last_error, grp)
    return _tune_dict(r)


# ---------------------------------------------------------------------------
# serving loop
# ---------------------------------------------------------------------------

def esc_server_create(grp: int, max_pending_updates: int, max_batches_per_call: int = 0) -> int:
    L = load()
    h = C.c_void_p()
    rc = L.esc_server_create(grp, int(max_pending_updates), int(max_batches_per_call), C.byref(h))
    if rc != 0:
        raise EscError(rc, "esc_server_create failed")
    return h.value


def esc_server_submit(srv: int, graph: int, ins_offsets=None, ins_members=None, ins_timestamps=None,
                      del_ids=None, out_ids: Optional[np.ndarray] = None, t_arrival_ns: int = 0) -> int:
    """Queue one request (host arrays; they are copied).  Returns the ticket,
    or -1 when the queue is full (ESC_ERR_BUSY).  ``out_ids`` (int32 numpy
    array) must stay alive until the request is collected."""
    L = load()
    b = esc_batch()
    b.graph = int(graph)
    po, ko = _ptr(ins_offsets, np.int64)
    pm, km = _ptr(ins_members, np.int32)
    pt, kt = _ptr(ins_timestamps, np.int64)
    pd, kd = _ptr(del_ids, np.int32)
    b.n_ins = (len(ins_offsets) - 1) if ins_offsets is not None and len(ins_offsets) else 0
    b.ins_offsets, b.ins_members, b.ins_timestamps = po, pm, pt
    b.n_del = len(del_ids) if del_ids is not None else 0
    b.del_ids = pd
    b.out_ins_ids = out_ids.ctypes.data if out_ids is not None and b.n_ins else None
    t = C.c_int64(-1)
    rc = L.esc_server_submit(srv, C.byref(b), int(t_arrival_ns), C.byref(t))
    if rc == ESC_ERR_BUSY:
        return -1
    if rc != 0:
        raise EscError(rc, "esc_server_submit failed")
    return int(t.value)


def esc_server_wait(srv: int, ticket: int) -> dict:
    """Block until the request is done; returns its record (status included)."""
    L = load()
    inf = esc_request_info()
    L.esc_server_wait(srv, int(ticket), C.byref(inf))
    return {k: getattr(inf, k) for k, _ in esc_request_info._fields_}


def esc_server_drain(srv: int) -> None:
    load().esc_server_drain(srv)


def esc_server_triads(srv: int, graph: int, triad_type: int, window: int = 0) -> np.ndarray:
    L = load()
    n = N_CLASSES[triad_type]
    out = np.zeros(n, np.uint64)
    rc = L.esc_server_triads(srv, int(graph), triad_type, int(window), out.ctypes.data, n)
    if rc != 0:
        raise EscError(rc, "esc_server_triads failed")
    return out


def esc_server_get_stats(srv: int) -> dict:
    L = load()
    s = esc_server_stats()
    L.esc_server_get_stats(srv, C.byref(s))
    return {k: getattr(s, k) for k, _ in esc_server_stats._fields_}


def esc_server_add_group(srv: int, grp: int) -> int:
    """Serve another group; returns the server-wide index of its graph 0."""
    L = load()
    first = C.c_int32(-1)
    rc = L.esc_server_add_group(srv, grp, C.byref(first))
    if rc != 0:
        raise EscError(rc, "esc_server_add_group failed")
    return int(first.value)


def esc_group_fits(shared: esc_config, graph_cfgs: Sequence[esc_config], reserve_bytes: int) -> bool:
    """Whether a group of this configuration fits the current device's free
    memory less reserve_bytes (nothing is allocated)."""
    L = load()
    arr = (esc_config * len(graph_cfgs))(*graph_cfgs)
    fits = C.c_int32(0)
    rc = L.esc_group_fits(C.byref(shared), len(graph_cfgs), arr, int(reserve_bytes), C.byref(fits))
    if rc != 0:
        raise EscError(rc, "esc_group_fits failed")
    return bool(fits.value)


def esc_server_destroy(srv: int) -> None:
    if srv:
        load().esc_server_destroy(srv)


def esc_count_static_noalloc(n_vertices: int, offsets, members, timestamps, families: int, delta: int,
                             out_counts, stream=None) -> None:
    """All triad counts of a static hypergraph whose arrays are CUDA tensors,
    written to ``out_counts`` (a CUDA int64/uint64 tensor of 129 entries),
    without any device allocation by the library."""
    L = load()

    def cuda_tensor(t, name, dtype, optional=False):
        if t is None and optional:
            return
        ok = (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and str(t.dtype) == dtype)
        if not ok:
            raise EscError(1, f"{name} must be a contiguous CUDA tensor of {dtype}")

    cuda_tensor(offsets, "offsets", "torch.int64")
    cuda_tensor(members, "members", "torch.int32")
    cuda_tensor(timestamps, "timestamps", "torch.int64", optional=True)
    if not (hasattr(out_counts, "is_cuda") and out_counts.is_cuda and out_counts.is_contiguous()
            and out_counts.element_size() == 8 and out_counts.numel() >= 129):
        raise EscError(1, "out_counts must be a contiguous CUDA tensor of at least 129 8-byte entries")
    po, ko = _ptr(offsets, np.int64)
    pm, km = _ptr(members, np.int32)
    pt, kt = _ptr(timestamps, np.int64)
    n_he = len(offsets) - 1
    rc = L.esc_count_static_noalloc(int(n_vertices), n_he, po, pm, pt, int(families), int(delta),
                                    out_counts.data_ptr(), _stream_ptr(stream))
    if rc != 0:
        raise EscError(rc, L.esc_last_error(None).decode())


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

def make_config(n_vertices: int, capacity_hyperedges: int, capacity_incidences: int,
                max_batch_hyperedges: int, max_batch_incidences: int, families: int,
                delta: int = 0, capacity_vertex_pairs: int = 0, debug: int = 0) -> esc_config:
    return esc_config(int(n_vertices), int(capacity_hyperedges), int(capacity_incidences),
                      int(max_batch_hyperedges), int(max_batch_incidences), int(families), int(delta), int(debug),
                      int(capacity_vertex_pairs))


class Graph:
    """One resident hypergraph (a handle from esc_create)."""

    def __init__(self, n_vertices: int, offsets=None, members=None, timestamps=None, *,
                 capacity_hyperedges: int, capacity_incidences: int, max_batch_hyperedges: int,
                 max_batch_incidences: int, families: int, delta: int = 0, stream=None,
                 capacity_vertex_pairs: int = 0, debug: int = 0):
        self.n_vertices = int(n_vertices)
        self.families = families
        self.delta = int(delta)
        self.cfg = make_config(n_vertices, capacity_hyperedges, capacity_incidences, max_batch_hyperedges,
                               max_batch_incidences, families, delta, capacity_vertex_pairs, debug)
        if offsets is None:
            offsets = np.zeros(1, np.int64)
            members = np.zeros(0, np.int32)
        self.h = esc_create(self.cfg, offsets, members, timestamps, stream)

    @classmethod
    def restore(cls, n_vertices: int, checkpoint: dict, *, capacity_hyperedges: int, capacity_incidences: int,
                max_batch_hyperedges: int, max_batch_incidences: int, families: int, delta: int = 0,
                stream=None) -> "Graph":
        """A graph holding ``checkpoint`` (an ``export()`` result) under its IDs."""
        self = cls.__new__(cls)
        self.n_vertices = int(n_vertices)
        self.families = families
        self.delta = int(delta)
        self.cfg = make_config(n_vertices, capacity_hyperedges, capacity_incidences, max_batch_hyperedges,
                               max_batch_incidences, families, delta)
        self.h = 0
        self.h = esc_restore(self.cfg, checkpoint["ids"], checkpoint["offsets"], checkpoint["members"],
                             checkpoint.get("timestamps"), stream)
        return self

    def export_h2h(self, s: int = 1) -> dict:
        return esc_export_h2h(self.h, s)

    def insert_with_ids(self, ids, offsets, members, timestamps=None) -> None:
        esc_insert_with_ids(self.h, ids, offsets, members, timestamps)

    def apply_batch(self, ins_offsets=None, ins_members=None, ins_timestamps=None, del_ids=None,
                    return_ids: bool = True) -> Optional[np.ndarray]:
        n_ins = (len(ins_offsets) - 1) if ins_offsets is not None and len(ins_offsets) else 0
        out = np.zeros(max(n_ins, 1), np.int32) if return_ids else None
        esc_apply_batch(self.h, ins_offsets, ins_members, ins_timestamps, del_ids, out)
        return out[:n_ins] if return_ids else None

    def triads(self, triad_type: int) -> np.ndarray:
        return esc_triads(self.h, triad_type, self.delta if triad_type == TRIAD_TEMPORAL else 0)

    def counts(self) -> dict:
        out = {}
        if self.families & FAMILY_HYPEREDGE:
            out["hyperedge"] = self.triads(TRIAD_HYPEREDGE)
        if self.families & (FAMILY_VERTEX | FAMILY_VERTEX12):
            out["vertex"] = self.triads(TRIAD_VERTEX)
        if self.families & FAMILY_TEMPORAL:
            out["temporal"] = self.triads(TRIAD_TEMPORAL)
        return out

    def local_triads(self, ids) -> dict:
        oh, ov, ot = esc_local_triads(self.h, ids)
        out = {}
        if self.families & FAMILY_HYPEREDGE:
            out["hyperedge"] = oh
        if self.families & FAMILY_VERTEX:
            out["vertex"] = ov
        if self.families & FAMILY_TEMPORAL:
            out["temporal"] = ot
        return out

    def export(self) -> dict:
        return esc_export(self.h, self.n_vertices)

    def stats(self) -> dict:
        return esc_last_stats(self.h)

    def set_profiling(self, on: bool = True) -> None:
        esc_set_profiling(self.h, on)

    def launch_count(self) -> int:
        return esc_launch_count(self.h)

    def autotune(self, ids, reps: int = 2) -> dict:
        return esc_autotune(self.h, ids, reps)

    def set_graph_launch(self, on: bool = True) -> None:
        esc_set_graph_launch(self.h, on)

    def set_split(self, rank: int, world: int) -> None:
        esc_set_split(self.h, rank, world)

    def update_members(self, ids, offsets, members) -> None:
        esc_update_members(self.h, ids, offsets, members)

    def close(self) -> None:
        if self.h:
            esc_destroy(self.h)
            self.h = 0

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
