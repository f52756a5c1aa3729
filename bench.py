#!/usr/bin/env python
"""Benchmark of the SPC hub-label path on GB300.

One step = one full pass of the path over the mixed pair of large graphs:
for R-MAT scale 20 (edge factor 8) and then the 256x256 grid with 10% of
its edges deleted, pspc_build (rank relabel, level-synchronous pull
construction, finalize) followed by pspc_query on 10^7 uniform (s,t)
pairs. Inputs are resident in device memory before the timed region; L2
is flushed (256 MiB write) before every build. Times are CUDA events on the
launching stream.

Prints one JSON line. ``value`` is label entries per second of the builds
(whole job: summed over ranks, divided by the slowest rank's time); query
throughput, both kernels' rooflines, an end-to-end pass through the C ABI
with host buffers, and the CPU oracle on a bounded sample are reported
beside it. ``--impl reference`` times the CPU oracle (the sequential
hub-pushing labeler) on a bounded sample of the same workload instead.

Multi-GPU: the path does not shard without an exchange step, so N ranks run
N independent replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ORACLE_SAMPLE_HUBS = 320  # bounded CPU sample: at most the 320 highest-ranked hubs per graph
ORACLE_BUILD_CAP_S = 12.0  # CPU build sample per graph, in seconds
ORACLE_QUERY_PAIRS = {"rmat20": 400, "grid256": 100_000}  # CPU query sample (first pairs of the set)
REFERENCE_BUDGET_S = 150.0  # whole --impl reference run, warm-up included

# A workload is one graph, or a list of graphs built one after another in
# every step.
WORKLOAD_GRAPHS = {"cfg3": ["rmat20", "grid256"]}
WORKLOAD_DESC = {
    "cfg3": ("Mixed pair: R-MAT scale 20 (1,048,576 vertices), edge factor 8, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
             "seed 1, symmetrised, self-loops and duplicates removed; and a 256x256 4-neighbour grid with 10% of "
             "edges deleted uniformly (seed 1), largest component kept; degree-descending rank with random "
             "tie-break (seed 3); per-graph index build plus 10^7 uniform random (s,t) pairs each (seed 2); "
             "uint64 counts with overflow flags"),
    "rmat16": ("R-MAT scale 16 (65,536 vertices), edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
               "seed 1, symmetrised, self-loops and duplicates removed, degree-descending rank "
               "(ties by id), int32 CSR; index build + uniform random (s,t) pairs (seed 2)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cfg3")
    ap.add_argument("--queries", type=int, default=10_000_000, help="query pairs per graph and step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cfg2-steps", type=int, default=10, help="timed passes of the R-MAT 16 extra figures")
    return ap.parse_args()


def graph_names(workload: str):
    return WORKLOAD_GRAPHS.get(workload, [workload])


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi sampling (100 ms) of SM clocks and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pspc_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 r[2:]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha(files) -> str:
    """Hash of a kernel's sources (a profile is stale once they change)."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2212_00977_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


LEVEL_SOURCES = ("pspc_level.cu", "pspc_level.cuh", "pspc_internal.cuh")
QUERY_SOURCES = ("pspc_query.cu", "pspc_internal.cuh")


def profiled_traffic(name: str, workload: str, sources):
    """DRAM bytes per unit (a level of the level kernels, a query call) from
    a committed ncu summary (profiles/<name>_<workload>.json), if it was
    taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", f"{name}_{workload}.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if kernel_source_sha(sources) != d.get("source_sha256"):
        return None
    return d.get("dram_bytes_per_unit")


def reduce_max(vals, dist, device):
    """Max over ranks of each value (times: the slowest rank sets the pace)."""
    if dist is None:
        return list(vals)
    import torch

    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rates(entries, queries, steps, world, t_build_ms, t_query_ms):
    """Whole-job throughput of N independent replicas: everything all ranks
    built (queried) divided by the slowest rank's time."""
    return (world * steps * entries / (t_build_ms / 1e3), world * steps * queries / (t_query_ms / 1e3))


def level_algorithmic_bytes(ls):
    """Bytes any pull implementation must move at one level: the CSR arcs of
    the active vertices (4 B), every pulled entry (hub 4 B + count 8 B) and
    every appended entry (12 B). The prune reads are not counted."""
    return 4 * ls["active_arcs"] + 12 * ls["raw_candidates"] + 12 * ls["entries"]


def query_algorithmic_bytes(sizes, pairs, dist_out):
    """Bytes of one query batch: per pair its 8-byte (s,t) and 11-byte
    answer, and for s != t the hub and distance words of both labels (6 B
    per entry) and, when reachable, the counts of at least one hub at the
    minimum on both sides (16 B)."""
    import numpy as np

    s = pairs[:, 0].astype(np.int64)
    t = pairs[:, 1].astype(np.int64)
    diff = s != t
    lab = (sizes[s] + sizes[t]).astype(np.int64)
    reach = diff & (dist_out != 0xFFFF)
    return int(19 * len(pairs) + 6 * lab[diff].sum() + 16 * reach.sum())


def cpu_build_baseline(g, rank, hubs=ORACLE_SAMPLE_HUBS, time_cap_s=ORACLE_BUILD_CAP_S):
    """The oracle's labeler on (at most) the `hubs` highest-ranked hubs,
    stopped after `time_cap_s`; returns (entries, seconds, hubs done)."""
    import oracle

    t0 = time.perf_counter()
    ix = oracle.OracleIndex(g, rank, max_hubs=hubs, time_cap_s=time_cap_s)
    dt = time.perf_counter() - t0
    return ix.entries, dt, ix.hubs_done


def cpu_query_baseline(g, pairs):
    """The oracle's SPC of the given pairs by breadth-first counting from
    each distinct source, sources in parallel on the host cores; returns
    (pairs, seconds, threads)."""
    import oracle

    t0 = time.perf_counter()
    _, _, _, th = oracle.spc_pairs(g, pairs)
    return len(pairs), time.perf_counter() - t0, th


def host_cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def run_reference(args):
    rank_id, _, world = dist_info()
    if rank_id != 0:
        return 0
    import pspc_inputs as P

    graphs = [(name,) + tuple(P.workload(name)[:2]) for name in graph_names(args.workload)]
    # Each step labels the top `hubs` hubs of every graph. The counts are
    # sized during the warm-up steps so that the whole run takes about
    # REFERENCE_BUDGET_S: the labeler's time grows about with the square of
    # the hubs it has done (each new hub's search queries the labels built
    # so far).
    per_step = max(0.5, min(12.0, REFERENCE_BUDGET_S / max(args.warmup + args.steps, 1))) / len(graphs)
    hubs = {name: 32 for name, _, _ in graphs}
    for _ in range(max(args.warmup, 1)):
        for name, g, rank in graphs:
            _, t, _ = cpu_build_baseline(g, rank, hubs=hubs[name], time_cap_s=0)
            h = hubs[name]
            hubs[name] = int(max(8, min(ORACLE_SAMPLE_HUBS, 4 * h, h * (per_step / max(t, 1e-3)) ** 0.5)))
    ent, times = 0, []
    for _ in range(args.steps):
        e_step, t_step = 0, 0.0
        for name, g, rank in graphs:
            e, dt, _ = cpu_build_baseline(g, rank, hubs=hubs[name], time_cap_s=0)
            e_step += e
            t_step += dt
        ent = e_step
        times.append(t_step)
    T = sum(times)
    value = ent * len(times) / T
    sample = ("hub-pushing labeler (C, 1 thread) over the highest-ranked hubs of each graph: "
              + ", ".join(f"{hubs[n]} of {n}" for n, _, _ in graphs) + f"; {ent} label entries per step")
    line = {"impl": "reference", "metric": "label entries/s (index build)", "value": value, "unit": "entries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload), "sample": sample},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Workload:
    """The graphs of a workload with their inputs resident on the device,
    and the timed pass of the path over them."""

    def __init__(self, names, queries, dev):
        import torch

        import pspc_inputs as P

        self.torch = torch
        self.dev = dev
        self.W = []
        for name in names:
            g, rank, pairs_fn = P.workload(name)
            pairs = pairs_fn(queries)
            q = len(pairs)
            self.W.append({"name": name, "g": g, "rank": rank, "pairs": pairs, "q": q,
                           "rp": torch.from_numpy(g.row_ptr).to(dev), "col": torch.from_numpy(g.col).to(dev),
                           "rk": torch.from_numpy(rank).to(dev), "pairs_d": torch.from_numpy(pairs).to(dev),
                           "od": torch.empty(q, dtype=torch.uint16, device=dev),
                           "oc": torch.empty(q, dtype=torch.uint64, device=dev),
                           "of": torch.empty(q, dtype=torch.uint8, device=dev)})
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)
        self.qbytes = {}

    def one(self, w, keep=False):
        """Build one graph's index, then answer its pairs (CUDA events on
        the launching stream; L2 flushed first)."""
        import paper_2212_00977_gb300 as pspc

        torch, stream = self.torch, self.stream
        self.flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = pspc.Index.build(w["g"].n, w["rp"], w["col"], w["rk"], stream=stream)
        e1.record(stream)
        ix.query(w["pairs_d"], w["od"], w["oc"], w["of"], stream=stream)
        e2.record(stream)
        e2.synchronize()
        r = {"build_ms": e0.elapsed_time(e1), "query_ms": e1.elapsed_time(e2), "st": ix.stats(),
             "ls": ix.level_stats()}
        if keep:
            r["ix"] = ix
        else:
            ix.free()
        return r

    def step(self):
        return [self.one(w) for w in self.W]

    def warm(self, warmup):
        """Warm-up passes; the first also fixes each graph's query bytes
        (label sizes of the finished index and the answers)."""
        for w in self.W:
            r = self.one(w, keep=True)
            sizes = r["ix"].label_sizes()
            self.qbytes[w["name"]] = query_algorithmic_bytes(sizes, w["pairs"], w["od"].cpu().numpy())
            r["ix"].free()
        for _ in range(max(warmup - 1, 0)):
            self.step()

    def summary(self, res, peak, peak_kind, workload):
        """Per-graph figures and the two rooflines of timed passes `res`."""
        K = len(res)
        per_graph = {}
        kb = kms = kl = qb = qms = 0.0
        for gi, w in enumerate(self.W):
            b = sum(level_algorithmic_bytes(l) for st in res for l in st[gi]["ls"])
            t = sum(l["kernel_ms"] for st in res for l in st[gi]["ls"])
            nl = sum(1 for st in res for l in st[gi]["ls"] if l["kernel_ms"] > 0)
            bq = self.qbytes[w["name"]] * K
            tq = sum(st[gi]["query_ms"] for st in res)
            tb = sum(st[gi]["build_ms"] for st in res)
            kb, kms, kl, qb, qms = kb + b, kms + t, kl + nl, qb + bq, qms + tq
            r = res[-1][gi]
            per_graph[w["name"]] = {
                "n": w["g"].n, "arcs": w["g"].arcs, "entries": r["st"]["entries"], "levels": r["st"]["levels"],
                "overflow_entries": r["st"]["overflow_entries"], "queries": w["q"],
                "build_ms": tb / K, "query_ms": tq / K,
                "entries_per_s": r["st"]["entries"] * K / (tb / 1e3), "queries_per_s": w["q"] * K / (tq / 1e3),
                "k_level_ms": t / K, "k_level_gbs": b / (t / 1e3) / 1e9 if t else 0.0,
                "query_gbs": bq / (tq / 1e3) / 1e9 if tq else 0.0, "landmark_ms": r["st"]["landmark_ms"]}
        achieved = kb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
        achieved_q = qb / (qms / 1e3) / 1e9 if qms > 0 else 0.0
        traffic = profiled_traffic("k_level", workload, LEVEL_SOURCES)
        traffic_q = profiled_traffic("k_query", workload, QUERY_SOURCES)
        # achieved: algorithmic bytes / device time; traffic: DRAM bytes of
        # one unit from the committed ncu summary (null when the kernel
        # sources changed since), and the DRAM rate it implies
        roof = {"kernel": "level kernels: pull gather + count merge + prune + append", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                "peak_kind": peak_kind, "traffic": traffic, "traffic_unit": "one level",
                "dram_gbs": (traffic * kl / (kms / 1e3) / 1e9) if (traffic and kms) else None,
                "bytes_per_step": kb / K, "kernel_ms_per_step": kms / K, "levels_per_step": kl / K}
        roof_q = {"kernel": "query call: source grouping + merge-join (Eq. (1)-(2))", "bound": "hbm",
                  "achieved": achieved_q, "peak": peak, "unit": "GB/s", "frac": achieved_q / peak if peak else None,
                  "peak_kind": peak_kind, "traffic": traffic_q, "traffic_unit": "one query call of one graph",
                  "dram_gbs": (traffic_q * len(self.W) * K / (qms / 1e3) / 1e9) if (traffic_q and qms) else None,
                  "bytes_per_step": qb / K, "ms_per_step": qms / K, "calls_per_step": len(self.W)}
        return per_graph, roof, roof_q


def run_ours(args):
    import torch

    import paper_2212_00977_gb300 as pspc

    rank_id, local_rank, world = dist_info()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    pspc.load()

    names = graph_names(args.workload)
    wl = Workload(names, args.queries, dev)
    W = wl.W
    wl.warm(args.warmup)
    sampler = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    res = [wl.step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()

    K = args.steps
    entries = sum(r["st"]["entries"] for r in res[-1])
    q_step = sum(w["q"] for w in W)
    T_build = sum(r["build_ms"] for st in res for r in st)
    T_query = sum(r["query_ms"] for st in res for r in st)
    T_build, T_query = reduce_max([T_build, T_query], dist, dev)
    value, qps = whole_job_rates(entries, q_step, K, world, T_build, T_query)
    launches_per_step = sum(r["st"]["kernel_launches"] + r["st"]["query_kernel_launches"] for r in res[-1])
    peak, peak_kind = measured_peak_hbm()
    per_graph, roof, roof_q = wl.summary(res, peak, peak_kind, args.workload)

    line = {"metric": "label entries/s (index build)", "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": (T_build + T_query) / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC.get(args.workload, args.workload), "graphs": names,
                       "queries_per_step": q_step, "l2": "flushed: 256 MiB device write before every build",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "build_ms": T_build / K, "query_ms": T_query / K, "queries_per_s": qps, "entries": entries,
            "per_graph": per_graph, "roofline": roof, "roofline_query": roof_q,
            "gpu_launches": launches_per_step * K, "clocks": clocks}

    if rank_id == 0 and world == 1 and args.workload == "cfg3" and args.cfg2_steps > 0:
        # the R-MAT 16 workload (10^6 pairs) as extra figures, outside the
        # timed region of the line's value
        w2 = Workload(["rmat16"], 1_000_000, dev)
        w2.warm(3)
        r2 = [w2.step() for _ in range(args.cfg2_steps)]
        pg2, roof2, roofq2 = w2.summary(r2, peak, peak_kind, "rmat16")
        line["cfg2"] = {"workload": WORKLOAD_DESC["rmat16"] + ", 10^6 pairs", "steps": args.cfg2_steps,
                        "warmup": 3, **pg2["rmat16"], "roofline": roof2, "roofline_query": roofq2}
        del w2
    if rank_id == 0 and world == 1 and args.e2e_steps > 0:
        # end to end through the public API with host buffers: the CSR,
        # rank and pairs are copied in and the answers out inside the calls
        tb = tq = 0.0
        for _ in range(args.e2e_steps):
            for w in W:
                wl.flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ix = pspc.Index.from_graph(w["g"], w["rank"])
                t1 = time.perf_counter()
                d, c, f = ix.query(w["pairs"])
                t2 = time.perf_counter()
                ix.free()
                tb += t1 - t0
                tq += t2 - t1
        h2d = sum(w["g"].row_ptr.nbytes + w["g"].col.nbytes + w["rank"].nbytes + w["pairs"].nbytes for w in W)
        d2h = q_step * (2 + 8 + 1)
        E = args.e2e_steps
        line["e2e"] = {"value": entries * E / tb, "unit": "entries/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "queries_per_s": q_step * E / tq, "step_s": (tb + tq) / E}
    if rank_id == 0 and world == 1 and not args.no_cpu_baseline:
        eb = tbs = 0.0
        done = []
        for w in W:
            e, dt, h = cpu_build_baseline(w["g"], w["rank"])
            eb, tbs = eb + e, tbs + dt
            done.append(f"{h} hubs of {w['name']} ({e} entries, {dt:.1f} s)")
        line["cpu_baseline"] = {
            "value": eb / tbs, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": "hub-pushing labeler (C, 1 thread) over the highest-ranked hubs of each graph, stopped "
                      f"after {ORACLE_BUILD_CAP_S:.0f} s per graph: " + "; ".join(done)}
        nq = tqs = 0.0
        qdone, threads = [], 1
        for w in W:
            k = min(w["q"], ORACLE_QUERY_PAIRS.get(w["name"], 10_000))
            m, dt, threads = cpu_query_baseline(w["g"], w["pairs"][:k])
            nq, tqs = nq + m, tqs + dt
            qdone.append(f"{m} pairs of {w['name']} in {dt:.1f} s")
        line["cpu_baseline_query"] = {
            "value": nq / tqs, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "cpu": host_cpu_model(), "nproc": os.cpu_count(),
            "sample": "SPC by breadth-first path counting from each distinct source (the definition), sources "
                      "in parallel on all host cores, over the first pairs of each graph's set: "
                      + "; ".join(qdone)}
    if rank_id == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """512 Barabasi-Albert graphs of uneven size (n ~ U[500, 20000],
    m ~ U{2..8}): one batched build and 10^5 queries per graph answered in
    one CUDA-graph replay, against the same work one graph at a time."""
    import numpy as np
    import torch

    import paper_2212_00977_gb300 as pspc
    import pspc_inputs as P
    from paper_2212_00977_gb300 import autotune

    count = 512
    qper = 100_000
    workers = min(16, os.cpu_count() or 1)
    batch = P.ba_batch(count, workers=workers)  # host processes start before any GPU call
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pspc.load()
    stream = torch.cuda.current_stream(dev)
    dbatch = [(n, torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev), torch.from_numpy(rank).to(dev))
              for (n, rp, col, rank) in batch]
    ns = np.array([b[0] for b in batch], np.int64)
    base = np.concatenate([[0], np.cumsum(ns)])
    rng = np.random.default_rng(2)
    pairs_np = np.concatenate([(rng.integers(0, n, size=(qper, 2)) + base[i]).astype(np.int32)
                               for i, n in enumerate(ns)])
    pairs = torch.from_numpy(pairs_np).to(dev)
    q = len(pairs_np)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # autotune the build tables on the first 32 graphs, the query variant on the full index
    sample = dbatch[:32]
    opts = autotune.tune_build(lambda **o: pspc.Index.build_batch(sample, **o), int(ns[:32].sum()),
                               int(sum(int(b[1][-1].item()) for b in sample)))
    d = torch.empty(q, dtype=torch.uint16, device=dev)
    c = torch.empty(q, dtype=torch.uint64, device=dev)
    f = torch.empty(q, dtype=torch.uint8, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)

    def batched_build():
        return pspc.Index.build_batch(dbatch, stream=stream, **opts)

    ix = batched_build()
    qv = autotune.tune_query(ix, pairs[: min(q, 2_000_000)])
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ix.query_async(pairs, d, c, f, err, stream=side)
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ix.query_async(pairs, d, c, f, err, stream=side)
    ix.free()

    b_ms, q_ms = [], []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = batched_build()
        e1.record(stream)
        stream.synchronize()
        # re-capture on the new index (its arrays moved), then time the replay
        graph = torch.cuda.CUDAGraph()
        ix.set_query_group(qv)
        with torch.cuda.graph(graph, stream=side):
            ix.query_async(pairs, d, c, f, err, stream=side)
        torch.cuda.synchronize()
        e1b, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):  # replay() launches on the current stream
            e1b.record(side)
            graph.replay()
            e2.record(side)
        e2.synchronize()
        if it >= args.warmup:
            b_ms.append(e0.elapsed_time(e1))
            q_ms.append(e1b.elapsed_time(e2))
        st = ix.stats()
        if it < args.warmup + args.steps - 1:
            ix.free()
    entries = st["entries"]
    bd, bc, bf = d.clone(), c.clone(), f.clone()
    assert int(err.item()) == 0
    ix.free()

    # one graph at a time: build, then its queries (same answers required)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    single_build_ms = single_query_ms = 0.0
    same = True
    for i, (n, rp, col, rank) in enumerate(dbatch):
        t0.record(stream)
        ix1 = pspc.Index.build(n, rp, col, rank, stream=stream)
        t1.record(stream)
        t1.synchronize()
        single_build_ms += t0.elapsed_time(t1)
        sl = slice(i * qper, (i + 1) * qper)
        local = pairs[sl] - int(base[i])
        t0.record(stream)
        sd, sc, sf = ix1.query(local.contiguous(), stream=stream)
        t1.record(stream)
        t1.synchronize()
        single_query_ms += t0.elapsed_time(t1)
        same &= bool(torch.equal(sd, bd[sl]) and torch.equal(sc, bc[sl]) and torch.equal(sf, bf[sl]))
        ix1.free()
    K = args.steps
    line = {"metric": "label entries/s (index build)", "value": entries * K / (sum(b_ms) / 1e3),
            "unit": "entries/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": (sum(b_ms) + sum(q_ms)) / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "512 Barabasi-Albert graphs, n ~ U[500,20000], m ~ U{2..8}, seeds 1000+i, "
                                   "degree-descending rank; one batched build + 10^5 random pairs per graph "
                                   "in one CUDA-graph replay",
                       "vertices": int(ns.sum()), "queries_per_step": q, "build_opts": opts, "query_variant": qv,
                       "l2": "flushed: 256 MiB device write before every step"},
            "build_ms": sum(b_ms) / K, "query_ms": sum(q_ms) / K, "queries_per_s": q * K / (sum(q_ms) / 1e3),
            "entries": entries,
            "one_at_a_time": {"build_ms": single_build_ms, "query_ms": single_query_ms,
                              "build_speedup": single_build_ms / (sum(b_ms) / K),
                              "query_speedup": single_query_ms / (sum(q_ms) / K), "same_answers": same}}
    print(json.dumps(line), flush=True)
    return 0 if same else 1


def run_serve(args):
    """Resident R-MAT scale-20 index; Poisson arrivals (mean 2,000/s) of
    query sets sized log-uniform in [1, 4096]; 1% of the requests are builds
    of Barabasi-Albert graphs (n ~ log-uniform [10^3, 10^5], m ~ U{2..8})
    admitted by estimated label memory. Reports p50/p99 latency from arrival
    to result on the host, and query throughput."""
    import threading

    import numpy as np
    import torch

    import paper_2212_00977_gb300 as pspc
    import pspc_inputs as P
    from paper_2212_00977_gb300 import serve

    rate = 2000.0
    duration = 8.0
    workers = min(16, os.cpu_count() or 1)
    rng = np.random.default_rng(4)
    n_req = int(rate * duration * 1.2)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration]
    is_build = rng.random(len(arrivals)) < 0.01
    n_builds = int(is_build.sum())
    bn = np.exp(rng.uniform(np.log(1e3), np.log(1e5), size=n_builds)).astype(np.int64)
    bm = rng.integers(2, 9, size=n_builds)
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(workers) as pool:
        built = pool.map(P._ba_member, [(i, bn[i], bm[i], 5000 + i) for i in range(n_builds)])
    build_graphs = [(P.Graph(n, rp, col, "ba"), rank) for (_, n, rp, col, rank) in built]
    g, rank, _ = P.workload("rmat20")
    sizes = np.exp(rng.uniform(0, np.log(4096), size=len(arrivals))).astype(np.int64)
    pool_pairs = P.query_pairs(g.n, int(sizes.sum()) + 1, 2)

    torch.cuda.set_device(0)
    pspc.load()
    dev = torch.device("cuda", 0)
    ix = pspc.Index.build(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                          torch.from_numpy(rank).to(dev))
    srv = serve.SPCServer(max_batch_pairs=1 << 21)
    srv.add_index("rmat20", ix)
    # warm-up
    srv.submit_query("rmat20", pool_pairs[:4096]).wait(60)
    reqs_q, reqs_b = [], []
    t0 = time.perf_counter() + 0.2
    off = 0
    bi = 0
    resident_built = []

    def driver():
        nonlocal off, bi
        for k, a in enumerate(arrivals):
            at = t0 + a
            now = time.perf_counter()
            if at > now:
                time.sleep(at - now)
            if is_build[k]:
                gb, rb = build_graphs[bi]
                name = f"ba{bi}"
                reqs_b.append((name, srv.submit_build(name, gb, rb, arrival=at)))
                bi += 1
            else:
                sz = int(sizes[k])
                reqs_q.append(srv.submit_query("rmat20", pool_pairs[off:off + sz], arrival=at))
                off += sz

    done_builds = 0
    failed_builds = []
    stop_reaper = threading.Event()

    def reaper():
        # clients release a built index as soon as it is ready
        nonlocal done_builds
        k = 0
        while not (stop_reaper.is_set() and k >= len(reqs_b)):
            if k >= len(reqs_b):
                time.sleep(0.001)
                continue
            name, r = reqs_b[k]
            try:
                r.wait(600)
                done_builds += 1
                srv.drop_index(name)
            except Exception as e:  # reported, not fatal to the load
                failed_builds.append(repr(e))
            k += 1

    th = threading.Thread(target=driver)
    rp = threading.Thread(target=reaper)
    th.start()
    rp.start()
    th.join()
    for r in reqs_q:
        r.wait(600)
    stop_reaper.set()
    rp.join()
    t_end = max(r.finished for r in reqs_q)
    sst = srv.stats()
    srv.close()
    lat_ms = [1e3 * r.latency for r in reqs_q]
    blat_ms = [1e3 * r.latency for _, r in reqs_b if r.finished]
    pairs_total = int(sum(len(r.pairs) for r in reqs_q))
    wall = t_end - t0
    line = {"metric": "SPC queries/s served; p50/p99 query latency", "value": pairs_total / wall,
            "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * wall,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "resident R-MAT scale 20 index; Poisson arrivals mean 2000/s for 8 s; query sets "
                                   "log-uniform in [1,4096] pairs; 1% build requests of BA graphs n in [1e3,1e5] "
                                   "(log-uniform), m ~ U{2..8}, admitted by estimated label memory",
                       "requests": len(arrivals), "query_requests": len(reqs_q), "build_requests": len(reqs_b)},
            "p50_ms": serve.percentile(lat_ms, 50), "p99_ms": serve.percentile(lat_ms, 99),
            "p50_build_ms": serve.percentile(blat_ms, 50), "p99_build_ms": serve.percentile(blat_ms, 99),
            "builds_done": done_builds, "batches": srv.batches, "pairs": pairs_total,
            "requests_per_batch": sst["requests_per_batch"], "pairs_per_batch": pairs_total / max(sst["batches"], 1),
            "max_builds_running": sst["max_builds_running"], "builds_failed": failed_builds}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
