"""Autotuner for the SPC library's tuning knobs.

Picks, by timing on the device, the query variant (lanes per pair, staged
chunk size or by-source, ``pspc_set_query_group``) and the build's on-chip
table sizes, label-map kind and landmark count (``pspc_opts``). Results
never depend on these choices; only speed does. Choices are cached per
workload class (size and density buckets) for the life of the process.
"""
from __future__ import annotations

import math

QUERY_VARIANTS = (1, 16, 32, 64, 128, 256)  # 1 = by source (pspc.PSPC_QUERY_BY_SOURCE)
BUILD_VARIANTS = tuple(dict(cand_capacity=c, map_kind=m) for c in (2048, 4096, 8192) for m in (0, 2, 3))
LANDMARK_VARIANTS = (-1, 32, 64, 128)  # second stage: landmark count on top of the best tables

_cache: dict = {}


def _elapsed_ms(fn, reps: int) -> float:
    import torch

    fn()  # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def workload_class(n: int, arcs: int, entries: int = 0) -> tuple:
    """Bucket of a workload: log2 of the vertex count, of the average degree
    and (for queries) of the average label size."""
    avg_deg = arcs / max(n, 1)
    avg_lab = entries / max(n, 1)
    return (int(math.log2(max(n, 1))), int(math.log2(avg_deg + 1)), int(math.log2(avg_lab + 1)))


def tune_query(ix, pairs_dev, reps: int = 3, variants=QUERY_VARIANTS) -> int:
    """Time every query variant on ``pairs_dev`` (a device int32 [q,2]
    tensor), set the fastest on ``ix`` and return it."""
    import torch

    st = ix.stats()
    key = ("query",) + workload_class(st["n"], st["arcs"], st["entries"])
    if key not in _cache:
        q = pairs_dev.shape[0]
        d = torch.empty(q, dtype=torch.uint16, device=pairs_dev.device)
        c = torch.empty(q, dtype=torch.uint64, device=pairs_dev.device)
        f = torch.empty(q, dtype=torch.uint8, device=pairs_dev.device)
        timing = {}
        for v in variants:
            ix.set_query_group(v)
            timing[v] = _elapsed_ms(lambda: ix.query(pairs_dev, d, c, f), reps)
        _cache[key] = min(timing, key=timing.get)
    ix.set_query_group(_cache[key])
    return _cache[key]


def _fastest(build, variants, reps):
    timing = {}
    for i, opts in enumerate(variants):
        def once(o=opts):
            build(**o).free()

        try:
            timing[i] = _elapsed_ms(once, reps)
        except RuntimeError:
            continue  # a variant the device cannot run (e.g. shared memory)
    return dict(variants[min(timing, key=timing.get)])


def tune_build(build, n: int, arcs: int, reps: int = 1, variants=BUILD_VARIANTS,
               landmarks=LANDMARK_VARIANTS) -> dict:
    """``build(**opts)`` builds and returns an Index; time each table
    variant on it, then the landmark counts on top of the fastest, and
    return the fastest options (the probe indexes are freed)."""
    key = ("build",) + workload_class(n, arcs)
    if key not in _cache:
        best = _fastest(build, variants, reps)
        if landmarks:
            best = _fastest(build, tuple(dict(best, landmarks=k) for k in landmarks), reps)
        _cache[key] = best
    return dict(_cache[key])


def clear() -> None:
    _cache.clear()
