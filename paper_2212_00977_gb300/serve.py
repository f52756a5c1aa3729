"""Serving loop for SPC queries and index builds on one GPU.

Indexes stay resident in device memory. Requests arrive at any time:

* query requests (an index name and an int32 [k, 2] array of (s, t) pairs)
  are served with continuous batching: while one batch runs on the GPU, new
  requests queue up; when it finishes, every queued request (up to the batch
  capacity) forms the next batch. Each batch makes one stream-ordered
  launch per index it touches, on the query stream, through the library's
  staging buffers.
* build requests (a graph and its order) run on their own stream, so a
  build overlaps the query batches on the device. A build is admitted only
  when its estimated label memory fits the memory budget next to the
  resident indexes and the builds already running; otherwise it waits.

Latency is measured from a request's arrival time (given by the caller, or
the submit time) to the moment its result is visible on the host.
Results do not depend on batching: each query's answer is the answer of
pspc_query on that pair alone.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import Index, PSPCError


def estimate_index_bytes(n: int, arcs: int) -> int:
    """Conservative device footprint of a build: label entries are estimated
    as n * (10 + 4 * avg_degree * log2(n)) (above what R-MAT and
    Barabasi-Albert graphs produce), at 14 bytes in the index plus 12 in the
    build arena, plus 24 bytes per arc of working arrays."""
    import math

    avg_deg = arcs / max(n, 1)
    entries = n * (10 + 4 * avg_deg * math.log2(max(n, 2)))
    return int(entries * 26 + arcs * 24 + n * 64)


class Request:
    __slots__ = ("kind", "name", "pairs", "graph", "arrival", "done", "result", "error", "finished", "opts")

    def __init__(self, kind, name, arrival, pairs=None, graph=None, opts=None):
        self.kind = kind
        self.name = name
        self.pairs = pairs
        self.graph = graph
        self.opts = opts or {}
        self.arrival = arrival
        self.done = threading.Event()
        self.result = None
        self.error = None
        self.finished = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    def wait(self, timeout=None):
        if not self.done.wait(timeout):
            raise TimeoutError("request not served in time")
        if self.error is not None:
            raise self.error
        return self.result


class SPCServer:
    def __init__(self, device: int = 0, max_batch_pairs: int = 1 << 21, memory_budget: int | None = None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.max_batch = int(max_batch_pairs)
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(memory_budget if memory_budget is not None else free * 0.8)
        # Queries get the high-priority stream. Builds launch their level
        # kernel one CTA per vertex (granular), so every finished vertex frees
        # an SM slot that a pending query block takes first, and their off-chip
        # pass keeps to one CTA per SM: a running build never holds the SMs
        # for a whole level.
        self.q_stream = torch.cuda.Stream(self.device, priority=-1)
        self.b_stream = torch.cuda.Stream(self.device, priority=0)
        self.pairs_h = torch.empty((self.max_batch, 2), dtype=torch.int32, pin_memory=True)
        self.dist_h = torch.empty(self.max_batch, dtype=torch.uint16, pin_memory=True)
        self.cnt_h = torch.empty(self.max_batch, dtype=torch.uint64, pin_memory=True)
        self.ovf_h = torch.empty(self.max_batch, dtype=torch.uint8, pin_memory=True)
        self.pairs_d = torch.empty((self.max_batch, 2), dtype=torch.int32, device=self.device)
        self.dist_d = torch.empty(self.max_batch, dtype=torch.uint16, device=self.device)
        self.cnt_d = torch.empty(self.max_batch, dtype=torch.uint64, device=self.device)
        self.ovf_d = torch.empty(self.max_batch, dtype=torch.uint8, device=self.device)
        self.err_d = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.indexes: dict[str, tuple[Index, int]] = {}
        self.reserved = 0  # bytes of builds admitted and running
        self.lock = threading.Condition()
        self.qq: collections.deque[Request] = collections.deque()
        self.bq: collections.deque[Request] = collections.deque()
        self.stop = False
        self.batches = 0
        self.batch_pairs = 0
        self.threads = [threading.Thread(target=self._query_loop, daemon=True),
                        threading.Thread(target=self._build_loop, daemon=True)]
        for t in self.threads:
            t.start()

    # --- public API -------------------------------------------------------
    def add_index(self, name: str, ix: Index) -> None:
        # The register-only query variant needs no shared memory, so its
        # blocks fit on SMs whose shared memory a running build fills.
        ix.set_query_group(32)
        st = ix.stats()
        with self.lock:
            self.indexes[name] = (ix, int(st["index_bytes"]))
            self.lock.notify_all()

    def drop_index(self, name: str) -> None:
        with self.lock:
            ix, _ = self.indexes.pop(name)
            self.lock.notify_all()
        ix.free()

    def resident_bytes(self) -> int:
        with self.lock:
            return sum(b for _, b in self.indexes.values())

    def submit_query(self, name: str, pairs: np.ndarray, arrival: float | None = None) -> Request:
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        if len(p) > self.max_batch:
            raise ValueError("query set larger than the batch capacity")
        r = Request("query", name, time.perf_counter() if arrival is None else arrival, pairs=p)
        with self.lock:
            self.qq.append(r)
            self.lock.notify_all()
        return r

    def submit_build(self, name: str, graph, rank, arrival: float | None = None, **opts) -> Request:
        r = Request("build", name, time.perf_counter() if arrival is None else arrival, graph=(graph, rank),
                    opts=opts)
        with self.lock:
            self.bq.append(r)
            self.lock.notify_all()
        return r

    def close(self) -> None:
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in self.threads:
            t.join()

    # --- workers ------------------------------------------------------------
    def _query_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                while not self.qq and not self.stop:
                    self.lock.wait()
                if self.stop and not self.qq:
                    return
                batch, total = [], 0
                while self.qq and total + len(self.qq[0].pairs) <= self.max_batch:
                    r = self.qq.popleft()
                    batch.append(r)
                    total += len(r.pairs)
                groups = collections.OrderedDict()
                for r in batch:
                    groups.setdefault(r.name, []).append(r)
                known = {name: self.indexes.get(name) for name in groups}
            self._run_batch(groups, known, total)

    def _run_batch(self, groups, known, total):
        torch = self.torch
        pos = 0
        spans = []  # (index, [(request, start)], start, end)
        for name, reqs in groups.items():
            ent = known.get(name)
            start = pos
            placed = []
            for r in reqs:
                if ent is None:
                    r.error = KeyError(f"no resident index {name!r}")
                    continue
                p = r.pairs
                if len(p) and (p.min() < 0 or p.max() >= ent[0].n):
                    r.error = PSPCError(1, "pspc_query")  # vertex id outside [0, n)
                    continue
                k = len(p)
                self.pairs_h[pos:pos + k].numpy()[:] = p
                placed.append((r, pos))
                pos += k
            if placed:
                spans.append((ent[0], placed, start, pos))
        if pos:
            with torch.cuda.stream(self.q_stream):
                self.pairs_d[:pos].copy_(self.pairs_h[:pos], non_blocking=True)
                for ix, placed, a, b in spans:
                    ix.query_async(self.pairs_d[a:b], self.dist_d[a:b], self.cnt_d[a:b], self.ovf_d[a:b],
                                   self.err_d, stream=self.q_stream)
                self.dist_h[:pos].copy_(self.dist_d[:pos], non_blocking=True)
                self.cnt_h[:pos].copy_(self.cnt_d[:pos], non_blocking=True)
                self.ovf_h[:pos].copy_(self.ovf_d[:pos], non_blocking=True)
            self.q_stream.synchronize()
        now = time.perf_counter()
        for ix, placed, a, b in spans:
            for r, off in placed:
                k = len(r.pairs)
                r.result = (self.dist_h[off:off + k].numpy().copy(), self.cnt_h[off:off + k].numpy().copy(),
                            self.ovf_h[off:off + k].numpy().copy())
        for reqs in groups.values():
            for r in reqs:
                r.finished = now
                r.done.set()
        self.batches += 1
        self.batch_pairs += pos

    def _build_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                while not self.bq and not self.stop:
                    self.lock.wait()
                if self.stop and not self.bq:
                    return
                r = self.bq.popleft()
                g, rank = r.graph
                need = estimate_index_bytes(g.n, g.arcs)
                # admission: wait until the estimate fits next to what is resident
                while (sum(b for _, b in self.indexes.values()) + self.reserved + need > self.budget
                       and not self.stop and self.reserved > 0):
                    self.lock.wait()
                if sum(b for _, b in self.indexes.values()) + need > self.budget and self.reserved == 0:
                    r.error = MemoryError("build does not fit the memory budget")
                    r.finished = time.perf_counter()
                    r.done.set()
                    continue
                self.reserved += need
            try:
                opts = dict(r.opts)
                opts.setdefault("granular", True)
                ix = Index.from_graph(g, rank, stream=self.b_stream, **opts)
                self.add_index(r.name, ix)
                r.result = ix.stats()
            except Exception as e:  # surfaced to the caller through wait()
                r.error = e
            finally:
                with self.lock:
                    self.reserved -= need
                    self.lock.notify_all()
                r.finished = time.perf_counter()
                r.done.set()


def percentile(xs, p: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), p)) if len(xs) else float("nan")
