"""Serving: continuously batched queries and overlapping builds give every
request exactly the answer the oracle gives, and the answer it gets alone;
builds are admitted by their estimated memory, wait for it when it is taken,
and fail at once only when they could never fit."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import oracle
import pspc_inputs as P
from tests import _graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as pspc
    from paper_2212_00977_gb300 import serve

    pspc.load()
    return torch, pspc, serve


def test_results_same_alone_and_in_the_mix(env):
    torch, pspc, serve = env
    srv = serve.SPCServer(max_batch_pairs=1 << 16)
    try:
        ga, ra, _ = P.workload("rmat12_ef16")
        gb, rb, _ = P.workload("ba2000")
        A = pspc.Index.from_graph(ga, ra)
        B = pspc.Index.from_graph(gb, rb)
        srv.add_index("A", A)
        srv.add_index("B", B)
        rng = np.random.default_rng(1)
        reqs = []
        # builds that overlap the query traffic
        gc = G.grid(30)
        gd = P.barabasi_albert(3000, 3, 11)
        bc = srv.submit_build("C", gc, G.random_rank(gc.n, 2))
        bd = srv.submit_build("D", gd, G.degree_rank(gd))

        def client(seed):
            r2 = np.random.default_rng(seed)
            for _ in range(60):
                name, g = ("A", ga) if r2.random() < 0.6 else ("B", gb)
                k = int(np.exp(r2.uniform(0, np.log(4096))))
                pairs = r2.integers(0, g.n, size=(k, 2)).astype(np.int32)
                reqs.append((name, pairs, srv.submit_query(name, pairs)))
                time.sleep(r2.exponential(0.0005))

        threads = [threading.Thread(target=client, args=(s,)) for s in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        bc.wait(120)
        bd.wait(120)
        for name, g in (("C", gc), ("D", gd)):
            pairs = rng.integers(0, g.n, size=(3000, 2)).astype(np.int32)
            reqs.append((name, pairs, srv.submit_query(name, pairs)))
        # an out-of-range request fails alone, without spoiling its batch
        bad = srv.submit_query("A", np.array([[0, ga.n]], np.int32))
        good = srv.submit_query("A", np.array([[0, 1]], np.int32))
        with pytest.raises(pspc.PSPCError):
            bad.wait(60)
        good.wait(60)
        alone = {"A": A, "B": B, "C": srv.indexes["C"][0], "D": srv.indexes["D"][0]}
        # the oracle's index of every graph (C and D were built by the
        # server while the queries ran)
        orc = {"A": oracle.OracleIndex(ga, ra), "B": oracle.OracleIndex(gb, rb),
               "C": oracle.OracleIndex(gc, G.random_rank(gc.n, 2)), "D": oracle.OracleIndex(gd, G.degree_rank(gd))}
        for name, pairs, r in reqs:
            d, c, f = r.wait(60)
            od, oc, of, _ = orc[name].query(pairs)
            assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
            rd, rc, rf = alone[name].query(pairs)
            assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
        assert srv.batches < len(reqs)  # requests were batched
        assert srv.stats()["requests_per_batch"] > 1
        lat = [r.latency for _, _, r in reqs]
        assert serve.percentile(lat, 99) < 60
    finally:
        srv.close()


def test_build_waits_for_memory_then_runs(env):
    """A build whose estimate fits the budget, but not next to a resident
    index, waits (it neither fails nor starts) until that index is dropped,
    then runs; its answers equal the oracle's. Two builds that fit together
    run at the same time."""
    torch, pspc, serve = env
    ga, ra, _ = P.workload("ba2000")
    gb = P.barabasi_albert(3000, 3, 21)
    rb = G.degree_rank(gb)
    A = pspc.Index.from_graph(ga, ra)
    a_bytes = A.stats()["index_bytes"]
    need_b = serve.estimate_index_bytes(gb.n, gb.arcs)
    srv = serve.SPCServer(max_batch_pairs=1 << 13, memory_budget=a_bytes + need_b - 1)
    try:
        srv.add_index("A", A)
        rb_req = srv.submit_build("B", gb, rb)
        time.sleep(1.0)
        assert not rb_req.done.is_set() and rb_req.started is None  # waiting for memory
        # queries keep being served meanwhile
        d, c, f = srv.submit_query("A", np.array([[0, 1], [5, 7]], np.int32)).wait(60)
        od, oc, of, _ = oracle.OracleIndex(ga, ra).query(np.array([[0, 1], [5, 7]], np.int32))
        assert np.array_equal(d, od) and np.array_equal(c, oc)
        t_drop = time.perf_counter()
        srv.drop_index("A")
        rb_req.wait(120)
        assert rb_req.started >= t_drop
        pairs = np.random.default_rng(3).integers(0, gb.n, size=(5000, 2)).astype(np.int32)
        d, c, f = srv.submit_query("B", pairs).wait(60)
        od, oc, of, _ = oracle.OracleIndex(gb, rb).query(pairs)
        assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
    finally:
        srv.close()
    # two builds admitted together overlap
    srv = serve.SPCServer(max_batch_pairs=1 << 13, max_builds=2)
    try:
        g1, g2 = G.grid(60), G.grid(61)
        r1 = srv.submit_build("g1", g1, G.random_rank(g1.n, 1))
        r2 = srv.submit_build("g2", g2, G.random_rank(g2.n, 2))
        r1.wait(120)
        r2.wait(120)
        assert max(r1.started, r2.started) < min(r1.finished, r2.finished)
        assert srv.stats()["max_builds_running"] == 2
        for name, g, rk in (("g1", g1, G.random_rank(g1.n, 1)), ("g2", g2, G.random_rank(g2.n, 2))):
            pairs = np.random.default_rng(4).integers(0, g.n, size=(3000, 2)).astype(np.int32)
            d, c, f = srv.submit_query(name, pairs).wait(60)
            od, oc, of, _ = oracle.OracleIndex(g, rk).query(pairs)
            assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
    finally:
        srv.close()


def test_admission_rejects_a_build_that_cannot_fit(env):
    torch, pspc, serve = env
    srv = serve.SPCServer(max_batch_pairs=1 << 10, memory_budget=1 << 20)
    try:
        g = P.barabasi_albert(5000, 4, 3)
        r = srv.submit_build("big", g, G.degree_rank(g))
        with pytest.raises(MemoryError):
            r.wait(60)
        with pytest.raises(KeyError):
            srv.submit_query("nope", np.array([[0, 1]], np.int32)).wait(60)
    finally:
        srv.close()


def test_concurrent_builds_from_threads(env):
    """Builds of different graphs (different on-chip table plans) run at the
    same time from two threads on their own streams; every one succeeds and
    equals the oracle."""
    torch, pspc, serve = env
    graphs = [P.barabasi_albert(int(n), int(m), 40 + i) for i, (n, m) in
              enumerate(zip(np.linspace(600, 9000, 16), [2, 3, 4, 5, 6, 7, 8, 3] * 2))]
    ranks = [G.degree_rank(g) for g in graphs]
    results = [None] * len(graphs)

    def worker(idx):
        st = torch.cuda.Stream()
        for i in idx:
            ix = pspc.Index.from_graph(graphs[i], ranks[i], stream=st)
            results[i] = ix.export()
            ix.free()

    ts = [threading.Thread(target=worker, args=(list(range(j, len(graphs), 2)),)) for j in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for g, rk, got in zip(graphs, ranks, results):
        ref = oracle.OracleIndex(g, rk).export()
        for a, b in zip(got, (ref.off, ref.hub, ref.dist, ref.cnt, ref.ovf)):
            assert np.array_equal(a, b)
