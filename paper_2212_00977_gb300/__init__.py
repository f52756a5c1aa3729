"""Python binding of the GB300 SPC hub-label library (``libpspc.so``).

Argument marshalling only: every step of the index build and the queries
runs in the CUDA kernels behind the C ABI declared in ``include/pspc.h``.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
the library detects where each pointer lives and stages host buffers
itself. There is no CPU fallback: importing works without a GPU, but every
call fails loudly when the shared library or a CUDA device is missing.

Names follow the paper (PSPC, arXiv 2212.00977): an index holds, per vertex
v, the label L(v) of entries (hub w, sd(v,w), trough path count tau(v,w)).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_cuda_build", "libpspc.so")

PSPC_OK = 0
PSPC_QUERY_BY_SOURCE = 1
PSPC_QUERY_BY_SOURCE_HASH = 2
PSPC_E_INVAL = 1
PSPC_E_NOMEM = 2
PSPC_E_CUDA = 3
PSPC_E_DIST = 5
UNREACHED = 0xFFFF

_lib = None
_lock = threading.Lock()


class PSPCError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (status {code})")


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("cand_capacity", ctypes.c_int32), ("label_capacity", ctypes.c_int32),
                ("arena_entries", ctypes.c_int64), ("max_levels", ctypes.c_int32),
                ("verbose", ctypes.c_int32), ("map_kind", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("granular", ctypes.c_int32), ("landmarks", ctypes.c_int32), ("reduce_shell", ctypes.c_int32),
                ("paradigm", ctypes.c_int32), ("warp_levels", ctypes.c_int32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("rank", ctypes.c_void_p)]


class LevelStat(ctypes.Structure):
    _fields_ = [("raw_candidates", ctypes.c_int64), ("unique_candidates", ctypes.c_int64),
                ("entries", ctypes.c_int64), ("active_vertices", ctypes.c_int64),
                ("active_arcs", ctypes.c_int64), ("ms", ctypes.c_float), ("kernel_ms", ctypes.c_float),
                ("landmark_pruned", ctypes.c_int64), ("landmark_proven", ctypes.c_int64),
                ("offchip_vertices", ctypes.c_int64), ("offchip_ms", ctypes.c_float),
                ("routed_vertices", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("arcs", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("levels", ctypes.c_int32), ("device", ctypes.c_int32),
                ("index_bytes", ctypes.c_int64), ("overflow_entries", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("query_kernel_launches", ctypes.c_int64),
                ("graphs", ctypes.c_int32), ("build_ms", ctypes.c_float),
                ("landmarks", ctypes.c_int32), ("landmark_ms", ctypes.c_float), ("shell_vertices", ctypes.c_int64)]


# Every symbol include/pspc.h declares, with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "pspc_build": (ctypes.c_int, [ctypes.POINTER(Csr), _P, ctypes.POINTER(Opts), ctypes.POINTER(_P), _P]),
    "pspc_query": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "pspc_query_async": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "pspc_build_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Opts),
                                        ctypes.POINTER(_P), _P]),
    "pspc_export": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pspc_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "pspc_level_stats": (ctypes.c_int, [_P, ctypes.POINTER(LevelStat), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "pspc_set_query_group": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pspc_export_vertices": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "pspc_hub_column": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "pspc_query_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "pspc_landmarks": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), _P, _P]),
    "pspc_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32]),
    "pspc_free": (None, [_P]),
    "pspc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libpspc.so (built by ``build_lib.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def inject_alloc_failure(after: int, status: int = PSPC_E_NOMEM) -> None:
    """pspc_inject_alloc_failure: the library's next ``after`` device
    allocations succeed and later ones fail with ``status`` (PSPC_E_NOMEM
    or PSPC_E_CUDA); ``after`` < 0 removes the limit. For tests of the
    error paths."""
    rc = load().pspc_inject_alloc_failure(int(after), int(status))
    if rc != PSPC_OK:
        raise PSPCError(rc, "pspc_inject_alloc_failure")


def strerror(code: int) -> str:
    try:
        return load().pspc_strerror(int(code)).decode()
    except Exception:  # the library itself may be what is missing
        return f"status {code}"


def _ptr(a):
    """Raw address of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check_dtype(a, np_dtype, name):
    if isinstance(a, np.ndarray):
        if a.dtype != np_dtype:
            raise TypeError(f"{name} must be {np.dtype(np_dtype).name}, got {a.dtype}")
    elif hasattr(a, "dtype"):
        want = {np.int64: "torch.int64", np.int32: "torch.int32", np.uint16: "torch.uint16",
                np.uint64: "torch.uint64", np.uint8: "torch.uint8"}[np_dtype]
        if str(a.dtype) != want:
            raise TypeError(f"{name} must be {want}, got {a.dtype}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Index:
    """A built SPC hub-label index living on one GPU (owned by the library)."""

    def __init__(self, handle: int, n: int):
        self._h = handle
        self.n = n

    @classmethod
    def build(cls, n: int, row_ptr, col, rank, *, stream=None, cand_capacity=0, label_capacity=0,
              arena_entries=0, max_levels=0, verbose=False, map_kind=0, max_ctas=0,
              granular=False, landmarks=0, reduce_shell=False, paradigm=0, warp_levels=0) -> "Index":
        """pspc_build over a symmetric CSR (rows strictly ascending) and a
        rank permutation (0 = highest). ``reduce_shell`` builds on the
        2-core and answers peeled tree vertices through their roots;
        ``paradigm=1`` builds each level by push instead of pull."""
        lib = load()
        _check_dtype(row_ptr, np.int64, "row_ptr")
        _check_dtype(col, np.int32, "col")
        _check_dtype(rank, np.int32, "rank")
        g = Csr(int(n), _ptr(row_ptr), _ptr(col))
        o = Opts(int(cand_capacity), int(label_capacity), int(arena_entries), int(max_levels),
                 int(bool(verbose)), int(map_kind), int(max_ctas), int(bool(granular)), int(landmarks),
                 int(bool(reduce_shell)), int(paradigm), int(warp_levels))
        h = _P()
        rc = lib.pspc_build(ctypes.byref(g), _ptr(rank), ctypes.byref(o), ctypes.byref(h),
                            _stream_handle(stream))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_build")
        return cls(h.value, int(n))

    @classmethod
    def build_batch(cls, graphs, *, stream=None, cand_capacity=0, label_capacity=0, arena_entries=0,
                    max_levels=0, verbose=False, map_kind=0, max_ctas=0,
                    granular=False, landmarks=0, warp_levels=0) -> "Index":
        """pspc_build_batch over ``graphs`` = [(n, row_ptr, col, rank), ...]:
        one index over their disjoint union (graph g's vertex v has id
        base_g + v, base_g = sum of earlier n)."""
        lib = load()
        k = len(graphs)
        arr = (GraphDesc * max(k, 1))()
        keep = []
        for i, (n, rp, col, rank) in enumerate(graphs):
            _check_dtype(rp, np.int64, "row_ptr")
            _check_dtype(col, np.int32, "col")
            _check_dtype(rank, np.int32, "rank")
            keep.append((rp, col, rank))
            arr[i] = GraphDesc(int(n), _ptr(rp), _ptr(col), _ptr(rank))
        o = Opts(int(cand_capacity), int(label_capacity), int(arena_entries), int(max_levels),
                 int(bool(verbose)), int(map_kind), int(max_ctas), int(bool(granular)), int(landmarks),
                 0, 0, int(warp_levels))
        h = _P()
        rc = lib.pspc_build_batch(ctypes.cast(arr, ctypes.c_void_p), k, ctypes.byref(o), ctypes.byref(h),
                                  _stream_handle(stream))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_build_batch")
        return cls(h.value, int(sum(int(g[0]) for g in graphs)))

    def query_async(self, pairs, dist, count, overflow, err, *, stream=None) -> None:
        """pspc_query_async: enqueue the queries on ``stream`` (device
        tensors only; ``err`` a device int32 tensor of one element)."""
        _check_dtype(pairs, np.int32, "pairs")
        q = int(pairs.shape[0])
        rc = load().pspc_query_async(self._h, _ptr(pairs), q, _ptr(dist), _ptr(count), _ptr(overflow), _ptr(err),
                                     _stream_handle(stream))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_query_async")

    @classmethod
    def from_graph(cls, g, rank, **kw) -> "Index":
        """Build from a ``pspc_inputs.Graph`` (host arrays)."""
        return cls.build(g.n, g.row_ptr, g.col, np.ascontiguousarray(rank, dtype=np.int32), **kw)

    def query(self, pairs, dist=None, count=None, overflow=None, *, stream=None):
        """pspc_query. ``pairs`` int32[q,2]. Outputs are allocated like the
        input (numpy for numpy, torch on the same device for torch) unless
        given. Returns (dist uint16, count uint64, overflow uint8)."""
        lib = load()
        _check_dtype(pairs, np.int32, "pairs")
        q = int(pairs.shape[0]) if len(pairs.shape) == 2 else int(pairs.shape[0]) // 2
        if dist is None:
            if isinstance(pairs, np.ndarray):
                dist = np.empty(q, np.uint16)
                count = np.empty(q, np.uint64)
                overflow = np.empty(q, np.uint8)
            else:
                import torch

                dist = torch.empty(q, dtype=torch.uint16, device=pairs.device)
                count = torch.empty(q, dtype=torch.uint64, device=pairs.device)
                overflow = torch.empty(q, dtype=torch.uint8, device=pairs.device)
        rc = lib.pspc_query(self._h, _ptr(pairs), q, _ptr(dist), _ptr(count), _ptr(overflow),
                            _stream_handle(stream))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_query")
        return dist, count, overflow

    def set_query_group(self, lanes: int) -> None:
        """Query variant of pspc_query: 8/16/32 lanes per pair, 64/128/256
        staged chunk entries, PSPC_QUERY_BY_SOURCE (L(s) on chip for the
        pairs of each source: a position table when it fits, else a hash),
        PSPC_QUERY_BY_SOURCE_HASH (the hash form), or 0 = automatic."""
        rc = load().pspc_set_query_group(self._h, int(lanes))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_set_query_group")

    def stats(self) -> dict:
        s = Stats()
        rc = load().pspc_stats(self._h, ctypes.byref(s))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def landmarks(self) -> np.ndarray:
        """pspc_landmarks: uint16 [n, k] distances from each vertex to the k
        landmarks of its graph (0xFFFF = unreached or none); k = 0 when the
        build ran without the landmark filter."""
        lib = load()
        k = ctypes.c_int32()
        rc = lib.pspc_landmarks(self._h, ctypes.byref(k), None, None)
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_landmarks")
        out = np.empty((self.n, k.value), dtype=np.uint16)
        if k.value:
            rc = lib.pspc_landmarks(self._h, ctypes.byref(k), _ptr(out), None)
            if rc != PSPC_OK:
                raise PSPCError(rc, "pspc_landmarks")
        return out

    def landmark_vertices(self) -> np.ndarray:
        """pspc_landmarks: int32 [k] caller ids of the landmarks of a
        one-graph index (-1: none)."""
        lib = load()
        k = ctypes.c_int32()
        rc = lib.pspc_landmarks(self._h, ctypes.byref(k), None, None)
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_landmarks")
        out = np.full(k.value, -1, dtype=np.int32)
        if k.value:
            rc = lib.pspc_landmarks(self._h, ctypes.byref(k), None, _ptr(out))
            if rc != PSPC_OK:
                raise PSPCError(rc, "pspc_landmarks")
        return out

    def level_stats(self) -> list[dict]:
        lib = load()
        cnt = ctypes.c_int32()
        rc = lib.pspc_level_stats(self._h, None, 0, ctypes.byref(cnt))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_level_stats")
        arr = (LevelStat * max(cnt.value, 1))()
        rc = lib.pspc_level_stats(self._h, arr, cnt.value, ctypes.byref(cnt))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_level_stats")
        return [{f: getattr(arr[i], f) for f, _ in LevelStat._fields_} for i in range(cnt.value)]

    def export(self):
        """pspc_export to host numpy arrays: (off, hub, dist, cnt, ovf), by
        caller vertex id, labels in hub-rank order, hubs as caller ids."""
        E = self.stats()["entries"]
        off = np.empty(self.n + 1, np.int64)
        hub = np.empty(E, np.int32)
        dist = np.empty(E, np.uint16)
        cnt = np.empty(E, np.uint64)
        ovf = np.empty(E, np.uint8)
        rc = load().pspc_export(self._h, _ptr(off), _ptr(hub), _ptr(dist), _ptr(cnt), _ptr(ovf))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_export")
        return off, hub, dist, cnt, ovf

    def export_vertices(self, verts):
        """pspc_export_vertices: labels of the given caller vertices as
        (off, hub, dist, cnt, ovf) host arrays."""
        lib = load()
        v = np.ascontiguousarray(verts, dtype=np.int32)
        k = len(v)
        off = np.empty(k + 1, np.int64)
        rc = lib.pspc_export_vertices(self._h, _ptr(v), k, _ptr(off), None, None, None, None)
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_export_vertices")
        E = int(off[-1])
        hub = np.empty(E, np.int32)
        dist = np.empty(E, np.uint16)
        cnt = np.empty(E, np.uint64)
        ovf = np.empty(E, np.uint8)
        rc = lib.pspc_export_vertices(self._h, _ptr(v), k, _ptr(off), _ptr(hub), _ptr(dist), _ptr(cnt), _ptr(ovf))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_export_vertices")
        return off, hub, dist, cnt, ovf

    def label_sizes(self, verts=None) -> np.ndarray:
        """Entries of L(v) for the given caller vertices (all by default),
        through pspc_export_vertices with only the offsets requested."""
        lib = load()
        v = np.arange(self.n, dtype=np.int32) if verts is None else np.ascontiguousarray(verts, dtype=np.int32)
        off = np.empty(len(v) + 1, np.int64)
        rc = lib.pspc_export_vertices(self._h, _ptr(v), len(v), _ptr(off), None, None, None, None)
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_export_vertices")
        return np.diff(off)

    def hub_column(self, w: int):
        """pspc_hub_column: (dist, cnt, ovf) of hub w in every label."""
        d = np.empty(self.n, np.uint16)
        c = np.empty(self.n, np.uint64)
        f = np.empty(self.n, np.uint8)
        rc = load().pspc_hub_column(self._h, int(w), _ptr(d), _ptr(c), _ptr(f))
        if rc != PSPC_OK:
            raise PSPCError(rc, "pspc_hub_column")
        return d, c, f

    def free(self):
        if self._h:
            load().pspc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()
