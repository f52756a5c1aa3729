"""Serving loop for SPC queries and index builds on one GPU.

Indexes stay resident in device memory. Requests arrive at any time:

* query requests (an index name and an int32 [k, 2] array of (s, t) pairs)
  are served with continuous batching: the query thread takes every queued
  request that fits the batch capacity, copies their pairs into a pinned
  staging slot and launches the batch (one stream-ordered pspc_query_async
  per index it touches) on that slot's high-priority stream, without
  waiting for it. There are `slots` such slots (default 2), so batch k+1 is
  formed, copied in and launched while batch k still runs; a completion
  thread waits for each batch in launch order and hands every request its
  answers. Requests that arrive while batches are on the GPU join the next
  batch as soon as a slot frees up.
* build requests (a graph and its order) run on build worker threads, each
  with its own stream, so builds overlap each other and the query batches.
  A build is admitted by its estimated device footprint: it starts when
  the estimate fits the memory budget next to the resident indexes and the
  builds already running; otherwise it waits until a dropped index or a
  finished build frees enough, and it fails at once only when it could
  never fit (the estimate exceeds the whole budget).

Latency is measured from a request's arrival time (given by the caller, or
the submit time) to the moment its result is visible on the host. Results
do not depend on batching: each query's answer is the answer of pspc_query
on that pair alone (Eq. (1)-(2) over the resident index).
"""
from __future__ import annotations

import collections
import math
import threading
import time

import numpy as np

from . import Index, PSPCError


def estimate_index_bytes(n: int, arcs: int) -> int:
    """Conservative device footprint of a build: label entries are estimated
    as n * (10 + 4 * avg_degree * log2(n)) (above what R-MAT and
    Barabasi-Albert graphs produce), at 14 bytes in the index plus 12 in the
    build arena, plus 24 bytes per arc of working arrays."""
    avg_deg = arcs / max(n, 1)
    entries = n * (10 + 4 * avg_deg * math.log2(max(n, 2)))
    return int(entries * 26 + arcs * 24 + n * 64)


class Request:
    __slots__ = ("kind", "name", "pairs", "graph", "arrival", "done", "result", "error", "finished", "opts",
                 "need", "started")

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
        self.need = 0
        self.started = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    def wait(self, timeout=None):
        if not self.done.wait(timeout):
            raise TimeoutError("request not served in time")
        if self.error is not None:
            raise self.error
        return self.result


class _Slot:
    """Pinned host and device buffers of one batch in flight, its stream
    and the event that marks the batch's end."""

    def __init__(self, torch, device, cap):
        self.stream = torch.cuda.Stream(device, priority=-1)
        self.pairs_h = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True)
        self.dist_h = torch.empty(cap, dtype=torch.uint16, pin_memory=True)
        self.cnt_h = torch.empty(cap, dtype=torch.uint64, pin_memory=True)
        self.ovf_h = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
        self.pairs_d = torch.empty((cap, 2), dtype=torch.int32, device=device)
        self.dist_d = torch.empty(cap, dtype=torch.uint16, device=device)
        self.cnt_d = torch.empty(cap, dtype=torch.uint64, device=device)
        self.ovf_d = torch.empty(cap, dtype=torch.uint8, device=device)
        self.err_d = torch.zeros(1, dtype=torch.int32, device=device)
        self.event = torch.cuda.Event()
        self.spans = []      # (index, [(request, offset)]) of the batch in flight
        self.groups = None   # every request of the batch
        self.indexes = []    # indexes the batch reads (kept alive until it ends)


class SPCServer:
    def __init__(self, device: int = 0, max_batch_pairs: int = 1 << 21, memory_budget: int | None = None,
                 slots: int = 2, max_builds: int = 2):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.max_batch = int(max_batch_pairs)
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(memory_budget if memory_budget is not None else free * 0.8)
        # Queries get high-priority streams. Builds launch their level
        # kernel one CTA per vertex (granular), so every finished vertex frees
        # an SM slot that a pending query block takes first, and their off-chip
        # pass keeps to one CTA per SM: a running build never holds the SMs
        # for a whole level.
        self.slots = [_Slot(torch, self.device, self.max_batch) for _ in range(max(1, slots))]
        self.free_slots = collections.deque(range(len(self.slots)))
        self.inflight: collections.deque[int] = collections.deque()
        self.launching = None  # slot of the batch being staged
        self.indexes: dict[str, tuple[Index, int]] = {}
        self.retired: list[Index] = []  # dropped while a batch could still read them
        self.reserved = 0  # bytes of builds admitted and running
        self.lock = threading.Condition()
        self.qq: collections.deque[Request] = collections.deque()
        self.bq: list[Request] = []
        self.stop = False
        self.batches = 0
        self.batch_pairs = 0
        self.batch_requests = 0
        self.builds_running = 0
        self.max_builds_running = 0
        self.threads = [threading.Thread(target=self._query_loop, daemon=True),
                        threading.Thread(target=self._complete_loop, daemon=True)]
        self.threads += [threading.Thread(target=self._build_loop, daemon=True) for _ in range(max(1, max_builds))]
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
        """Remove a resident index. Its memory is released as soon as no
        batch in flight reads it, and waiting builds are reconsidered."""
        with self.lock:
            ix, _ = self.indexes.pop(name)
            busy = id(ix) in self._busy_indexes()
            if busy:
                self.retired.append(ix)
            self.lock.notify_all()
        if not busy:
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
        r.need = estimate_index_bytes(graph.n, graph.arcs)
        with self.lock:
            if r.need > self.budget:  # could never fit, even with nothing resident
                r.error = MemoryError("build does not fit the memory budget")
                r.finished = time.perf_counter()
                r.done.set()
                return r
            self.bq.append(r)
            self.lock.notify_all()
        return r

    def close(self) -> None:
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in self.threads:
            t.join()
        for ix in self.retired:
            ix.free()
        self.retired = []

    def stats(self) -> dict:
        with self.lock:
            return {"batches": self.batches, "batch_pairs": self.batch_pairs, "batch_requests": self.batch_requests,
                    "requests_per_batch": self.batch_requests / max(self.batches, 1),
                    "max_builds_running": self.max_builds_running}

    # --- query batches --------------------------------------------------------
    def _busy_indexes(self):
        """Indexes that a batch in flight, or the one being staged, reads
        (caller holds the lock)."""
        ks = list(self.inflight) + ([self.launching] if self.launching is not None else [])
        return {id(ix) for k in ks for ix in self.slots[k].indexes}

    def _query_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                while not self.qq or not self.free_slots:
                    if self.stop and not self.qq:
                        return
                    self.lock.wait()
                k = self.free_slots.popleft()
                self.launching = k
                batch, total = [], 0
                while self.qq and total + len(self.qq[0].pairs) <= self.max_batch:
                    r = self.qq.popleft()
                    batch.append(r)
                    total += len(r.pairs)
                groups = collections.OrderedDict()
                for r in batch:
                    groups.setdefault(r.name, []).append(r)
                known = {name: self.indexes.get(name) for name in groups}
                self.slots[k].indexes = [ent[0] for ent in known.values() if ent is not None]
            self._launch(k, groups, known)

    def _launch(self, k, groups, known):
        """Stage a batch in slot k and enqueue it; the completion thread
        delivers its answers."""
        torch = self.torch
        slot = self.slots[k]
        pos = 0
        spans = []
        for name, reqs in groups.items():
            ent = known.get(name)
            placed = []
            for r in reqs:
                if ent is None:
                    r.error = KeyError(f"no resident index {name!r}")
                    continue
                p = r.pairs
                if len(p) and (p.min() < 0 or p.max() >= ent[0].n):
                    r.error = PSPCError(1, "pspc_query")  # vertex id outside [0, n)
                    continue
                n = len(p)
                slot.pairs_h[pos:pos + n].numpy()[:] = p
                placed.append((r, pos))
                pos += n
            if placed:
                spans.append((ent[0], placed))
        slot.spans = spans
        slot.groups = groups
        slot.indexes = [ix for ix, _ in spans]
        if pos:
            with torch.cuda.stream(slot.stream):
                slot.pairs_d[:pos].copy_(slot.pairs_h[:pos], non_blocking=True)
                a = 0
                for ix, placed in spans:
                    b = a + sum(len(r.pairs) for r, _ in placed)
                    ix.query_async(slot.pairs_d[a:b], slot.dist_d[a:b], slot.cnt_d[a:b], slot.ovf_d[a:b],
                                   slot.err_d, stream=slot.stream)
                    a = b
                slot.dist_h[:pos].copy_(slot.dist_d[:pos], non_blocking=True)
                slot.cnt_h[:pos].copy_(slot.cnt_d[:pos], non_blocking=True)
                slot.ovf_h[:pos].copy_(slot.ovf_d[:pos], non_blocking=True)
                slot.event.record(slot.stream)
        with self.lock:
            self.inflight.append(k)
            self.launching = None
            self.batches += 1
            self.batch_pairs += pos
            self.batch_requests += sum(len(v) for v in groups.values())
            self.lock.notify_all()

    def _complete_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                while not self.inflight:
                    if self.stop and not self.qq and self.launching is None:
                        return
                    self.lock.wait()
                k = self.inflight[0]
            slot = self.slots[k]
            slot.event.synchronize()
            now = time.perf_counter()
            for ix, placed in slot.spans:
                for r, off in placed:
                    n = len(r.pairs)
                    r.result = (slot.dist_h[off:off + n].numpy().copy(), slot.cnt_h[off:off + n].numpy().copy(),
                                slot.ovf_h[off:off + n].numpy().copy())
            for reqs in slot.groups.values():
                for r in reqs:
                    r.finished = now
                    r.done.set()
            with self.lock:
                self.inflight.popleft()
                slot.spans, slot.groups, slot.indexes = [], None, []
                self.free_slots.append(k)
                still = self._busy_indexes()
                gone = [ix for ix in self.retired if id(ix) not in still]
                self.retired = [ix for ix in self.retired if id(ix) in still]
                self.lock.notify_all()
            for ix in gone:
                ix.free()

    # --- builds -----------------------------------------------------------------
    def _admissible(self):
        """The first queued build whose estimate fits now (caller holds the lock)."""
        resident = sum(b for _, b in self.indexes.values())
        for r in self.bq:
            if resident + self.reserved + r.need <= self.budget:
                return r
        return None

    def _build_loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device, priority=0)
        while True:
            with self.lock:
                while not self.stop:
                    r = self._admissible() if self.bq else None
                    if r is not None:
                        break
                    self.lock.wait()
                if self.stop:
                    for q in self.bq:  # never started: fail them
                        q.error = RuntimeError("server closed")
                        q.finished = time.perf_counter()
                        q.done.set()
                    self.bq = []
                    return
                self.bq.remove(r)
                self.reserved += r.need
                self.builds_running += 1
                self.max_builds_running = max(self.max_builds_running, self.builds_running)
            r.started = time.perf_counter()
            try:
                g, rank = r.graph
                opts = dict(r.opts)
                opts.setdefault("granular", True)
                ix = Index.from_graph(g, rank, stream=stream, **opts)
                self.add_index(r.name, ix)
                r.result = ix.stats()
            except Exception as e:  # surfaced to the caller through wait()
                r.error = e
            finally:
                with self.lock:
                    self.reserved -= r.need
                    self.builds_running -= 1
                    self.lock.notify_all()
                r.finished = time.perf_counter()
                r.done.set()


def percentile(xs, p: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), p)) if len(xs) else float("nan")
