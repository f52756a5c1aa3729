"""CPU oracle for the SPC 2-hop hub-label index and the SPC(s,t) query.

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package. It shares
no code with the CUDA library and never imports it.

Three independent implementations of the same result:

* :mod:`oracle.brute` -- the plain definition (trough shortest paths, the
  ESPC construction of Section "PSPC algorithm description from the
  Covering Side"), in Python with exact big integers, for tiny graphs.
* ``pspc_oracle.c`` via :class:`OracleIndex` -- the sequential hub-pushing
  labeler in rank order (HP-SPC, Section "Order Property"), the Eq. (1)-(2)
  merge-join query, breadth-first path counting, and the per-hub column
  check straight from the definition, all in C with uint64 counts wrapping
  mod 2^64 and an overflow flag set iff the exact value is >= 2^64. For the
  full-size workloads the same definitions run in parallel on the host
  cores: columns of many hubs (:func:`hub_columns`), a whole exported index
  checked column by column (:func:`check_columns`), and query answers by
  one breadth-first count per source (:func:`spc_pairs`).

``build_lib()`` compiles the C file with gcc into ``oracle/_oracle_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pspc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_oracle_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lib = None
_lock = threading.Lock()

UNREACHED = 0xFFFF


def build_lib(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP) if it is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=199309L", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_build.restype = P
        lib.orc_build.argtypes = [I64, P, P, P, I64, ctypes.c_double]
        lib.orc_free.argtypes = [P]
        for f in ("orc_entries", "orc_hubs_done"):
            getattr(lib, f).restype = I64
            getattr(lib, f).argtypes = [P]
        lib.orc_truncated.argtypes = [P]
        lib.orc_max_dist.argtypes = [P]
        lib.orc_seconds.restype = ctypes.c_double
        lib.orc_seconds.argtypes = [P]
        lib.orc_export.argtypes = [P, P, P, P, P, P]
        lib.orc_query.restype = ctypes.c_int
        lib.orc_query.argtypes = [P, P, I64, P, P, P]
        lib.orc_bfs_count.argtypes = [I64, P, P, ctypes.c_int32, P, P, P, P, P, ctypes.c_int32]
        lib.orc_hub_column.restype = ctypes.c_int
        lib.orc_hub_column.argtypes = [I64, P, P, P, ctypes.c_int32, P, P, P]
        lib.orc_hub_columns.restype = ctypes.c_int
        lib.orc_hub_columns.argtypes = [I64, P, P, P, P, I64, P, P, P]
        lib.orc_spc_pairs.restype = ctypes.c_int
        lib.orc_spc_pairs.argtypes = [I64, P, P, P, I64, P, P, P]
        lib.orc_check_columns.restype = I64
        lib.orc_check_columns.argtypes = [I64, P, P, P, P, I64, P, P, P, P, P, P, P, P, I64]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Labels:
    """An exported index: per vertex (caller ids) its entries by hub rank.

    ``off`` int64[n+1]; ``hub`` int32[E] (caller vertex ids); ``dist``
    uint16[E]; ``cnt`` uint64[E] (exact count mod 2^64); ``ovf`` uint8[E]
    (1 iff the exact count is >= 2^64).
    """

    def __init__(self, off, hub, dist, cnt, ovf):
        self.off, self.hub, self.dist, self.cnt, self.ovf = off, hub, dist, cnt, ovf

    @property
    def n(self) -> int:
        return len(self.off) - 1

    @property
    def entries(self) -> int:
        return int(self.off[-1])

    def of(self, v: int):
        a, b = int(self.off[v]), int(self.off[v + 1])
        return [(int(self.hub[i]), int(self.dist[i]), int(self.cnt[i]), int(self.ovf[i]))
                for i in range(a, b)]


class OracleIndex:
    """Sequential hub-pushing labeler (C). ``max_hubs`` limits the build to
    the highest-ranked hubs, which gives exactly the full index restricted
    to those hubs; ``time_cap_s`` stops early (``truncated``)."""

    def __init__(self, g, rank: np.ndarray, max_hubs: int = -1, time_cap_s: float = 0.0):
        lib = _load()
        self._lib = lib
        self.n = int(g.n)
        self._row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        self._col = np.ascontiguousarray(g.col, dtype=np.int32)
        self._rank = np.ascontiguousarray(rank, dtype=np.int32)
        if self.n and (self._rank.min() < 0 or self._rank.max() >= self.n
                       or np.bincount(self._rank, minlength=self.n).max() > 1):
            raise ValueError("rank must be a permutation of 0..n-1")
        h = lib.orc_build(self.n, _ptr(self._row_ptr), _ptr(self._col), _ptr(self._rank),
                          int(max_hubs), float(time_cap_s))
        if not h:
            raise MemoryError("oracle build failed (allocation or distance > 32767)")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    @property
    def entries(self) -> int:
        return int(self._lib.orc_entries(self._h))

    @property
    def hubs_done(self) -> int:
        return int(self._lib.orc_hubs_done(self._h))

    @property
    def truncated(self) -> bool:
        return bool(self._lib.orc_truncated(self._h))

    @property
    def seconds(self) -> float:
        return float(self._lib.orc_seconds(self._h))

    @property
    def max_dist(self) -> int:
        return int(self._lib.orc_max_dist(self._h))

    def export(self) -> Labels:
        E = self.entries
        off = np.empty(self.n + 1, np.int64)
        hub = np.empty(E, np.int32)
        dist = np.empty(E, np.uint16)
        cnt = np.empty(E, np.uint64)
        ovf = np.empty(E, np.uint8)
        self._lib.orc_export(self._h, _ptr(off), _ptr(hub), _ptr(dist), _ptr(cnt), _ptr(ovf))
        return Labels(off, hub, dist, cnt, ovf)

    def query(self, pairs: np.ndarray):
        """Eq. (1)-(2) for int32[q,2] caller-id pairs: (dist uint16 with
        0xFFFF = unreachable, cnt uint64, ovf uint8, threads used)."""
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        if p.size and (p.min() < 0 or p.max() >= self.n):
            raise ValueError("pair vertex out of range")
        q = len(p)
        d = np.empty(q, np.uint16)
        c = np.empty(q, np.uint64)
        f = np.empty(q, np.uint8)
        th = self._lib.orc_query(self._h, _ptr(p), q, _ptr(d), _ptr(c), _ptr(f))
        return d, c, f, int(th)


def bfs_count(g, s: int):
    """Breadth-first shortest-path counting from s: (dist int32, -1 when
    unreachable; cnt uint64 mod 2^64; ovf uint8)."""
    lib = _load()
    n = int(g.n)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    d = np.empty(n, np.int32)
    c = np.empty(n, np.uint64)
    f = np.empty(n, np.uint8)
    qbuf = np.empty(max(n, 1), np.int32)
    lib.orc_bfs_count(n, _ptr(rp), _ptr(col), int(s), _ptr(d), _ptr(c), _ptr(f), _ptr(qbuf),
                      None, 0)
    return d, c, f


def hub_column(g, rank: np.ndarray, w: int):
    """Entry of hub w in every label, from the definition: (dist uint16 with
    0xFFFF where v has no entry for w, cnt uint64, ovf uint8)."""
    lib = _load()
    n = int(g.n)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    rk = np.ascontiguousarray(rank, dtype=np.int32)
    d = np.empty(n, np.uint16)
    c = np.empty(n, np.uint64)
    f = np.empty(n, np.uint8)
    if lib.orc_hub_column(n, _ptr(rp), _ptr(col), _ptr(rk), int(w), _ptr(d), _ptr(c), _ptr(f)):
        raise MemoryError("hub column allocation failed")
    return d, c, f


def spc_pairs(g, pairs: np.ndarray):
    """SPC of int32[q,2] pairs by breadth-first path counting, one search
    per distinct source, sources in parallel on the host cores: (dist uint16
    with 0xFFFF = unreachable, cnt uint64, ovf uint8, threads used)."""
    lib = _load()
    n = int(g.n)
    p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    if p.size and (p.min() < 0 or p.max() >= n):
        raise ValueError("pair vertex out of range")
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    q = len(p)
    d = np.empty(q, np.uint16)
    c = np.empty(q, np.uint64)
    f = np.empty(q, np.uint8)
    th = lib.orc_spc_pairs(n, _ptr(rp), _ptr(col), _ptr(p), q, _ptr(d), _ptr(c), _ptr(f))
    if th < 0:
        raise MemoryError("spc_pairs allocation failed")
    return d, c, f, int(th)


def check_columns(g, rank: np.ndarray, hubs, off, hub, dist, cnt, ovf, max_bad: int = 16):
    """Compare an exported index (caller ids, labels in strictly increasing
    hub rank) with the definition, column by column for the given hubs, in
    parallel on the host cores: every entry the definition gives must be in
    the index with its distance, count and flag. Returns (mismatching (hub,
    vertex) pairs, entries the definition gives for these hubs, list of the
    first bad (hub, vertex)); with all hubs, an entry total equal to the
    index size means the index holds nothing else."""
    lib = _load()
    n = int(g.n)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    rk = np.ascontiguousarray(rank, dtype=np.int32)
    hs = np.ascontiguousarray(hubs, dtype=np.int32)
    arrs = [np.ascontiguousarray(a) for a in (off, hub, dist, cnt, ovf)]
    assert [a.dtype for a in arrs] == [np.int64, np.int32, np.uint16, np.uint64, np.uint8]
    bw = np.zeros(max_bad, np.int32)
    bv = np.zeros(max_bad, np.int32)
    ent = ctypes.c_int64()
    bad = lib.orc_check_columns(n, _ptr(rp), _ptr(col), _ptr(rk), _ptr(hs), len(hs), *[_ptr(a) for a in arrs],
                                ctypes.byref(ent), _ptr(bw), _ptr(bv), max_bad)
    if bad < 0:
        raise MemoryError("check_columns allocation failed")
    k = min(int(bad), max_bad)
    return int(bad), int(ent.value), list(zip(bw[:k].tolist(), bv[:k].tolist()))


def hub_columns(g, rank: np.ndarray, hubs):
    """hub_column for many hubs, in parallel on the host cores: arrays
    [len(hubs), n] of (dist uint16 with 0xFFFF where there is no entry,
    cnt uint64, ovf uint8)."""
    lib = _load()
    n = int(g.n)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    rk = np.ascontiguousarray(rank, dtype=np.int32)
    hs = np.ascontiguousarray(hubs, dtype=np.int32)
    d = np.empty((len(hs), n), np.uint16)
    c = np.empty((len(hs), n), np.uint64)
    f = np.empty((len(hs), n), np.uint8)
    if lib.orc_hub_columns(n, _ptr(rp), _ptr(col), _ptr(rk), _ptr(hs), len(hs), _ptr(d), _ptr(c), _ptr(f)) < 0:
        raise MemoryError("hub_columns allocation failed")
    return d, c, f
