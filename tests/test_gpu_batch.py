"""Batched builds and CUDA-graph queries: one build over many graphs of
uneven size gives, for every graph, exactly the oracle's index of that
graph alone; queries captured in a CUDA graph give the same answers as
pspc_query; the autotuner changes speed, never answers."""
from __future__ import annotations

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

    pspc.load()
    return torch, pspc


def _mixed_batch():
    out = []
    for (n, rp, col, rank) in P.ba_batch(12, n_range=(60, 900), m_range=(1, 6), seed=77):
        out.append(P.Graph(n, rp, col, "ba"))
    out += [G.path(7), G.grid(9), G.diamond_chain(66), G.random_tree(50, 3), G.cycle(12),
            P.csr_from_edges(1, np.zeros((0, 2), np.int64)), G.complete(6),
            P.csr_from_edges(5, np.array([(0, 1), (3, 4)]))]
    ranks = [G.degree_rank(g) if i % 2 else G.random_rank(g.n, i) for i, g in enumerate(out)]
    return out, ranks


@pytest.mark.parametrize("device", [True, False])
def test_batch_build_equals_oracle_per_graph(env, device):
    torch, pspc = env
    graphs, ranks = _mixed_batch()
    dev = torch.device("cuda:0")
    conv = (lambda a: torch.from_numpy(a).to(dev)) if device else (lambda a: a)
    ix = pspc.Index.build_batch([(g.n, conv(g.row_ptr), conv(g.col), conv(r)) for g, r in zip(graphs, ranks)])
    assert ix.stats()["graphs"] == len(graphs)
    base = np.concatenate([[0], np.cumsum([g.n for g in graphs])]).astype(np.int64)
    rng = np.random.default_rng(3)
    pairs_all, want = [], []
    for i, (g, r) in enumerate(zip(graphs, ranks)):
        ref_ix = oracle.OracleIndex(g, r)
        ref = ref_ix.export()
        off, hub, dist, cnt, ovf = ix.export_vertices(np.arange(base[i], base[i + 1], dtype=np.int32))
        assert np.array_equal(off, ref.off)
        assert np.array_equal(hub - base[i], ref.hub)
        assert np.array_equal(dist, ref.dist) and np.array_equal(cnt, ref.cnt) and np.array_equal(ovf, ref.ovf)
        p = rng.integers(0, g.n, size=(200, 2)).astype(np.int32)
        pairs_all.append((p + base[i]).astype(np.int32))
        want.append(ref_ix.query(p)[:3])
    d, c, f = ix.query(np.concatenate(pairs_all))
    rd = np.concatenate([w[0] for w in want])
    rc = np.concatenate([w[1] for w in want])
    rf = np.concatenate([w[2] for w in want])
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
    # pairs from two different graphs are unreachable
    cross = np.array([[base[0], base[1]], [base[3] + 1, base[2]]], np.int32)
    d, c, f = ix.query(cross)
    assert d.tolist() == [0xFFFF, 0xFFFF] and c.tolist() == [0, 0]


def test_batch_answers_equal_single_builds(env):
    torch, pspc = env
    batch = P.ba_batch(24, n_range=(500, 4000), m_range=(2, 8), seed=1000)
    ix = pspc.Index.build_batch(batch)
    base = np.concatenate([[0], np.cumsum([b[0] for b in batch])])
    rng = np.random.default_rng(9)
    for i, (n, rp, col, rank) in enumerate(batch):
        single = pspc.Index.build(n, rp, col, rank)
        p = rng.integers(0, n, size=(5000, 2)).astype(np.int32)
        a = single.query(p)
        b = ix.query((p + base[i]).astype(np.int32))
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        so = single.export()
        bo = ix.export_vertices(np.arange(base[i], base[i + 1], dtype=np.int32))
        assert np.array_equal(so[0], bo[0]) and np.array_equal(so[1], bo[1] - base[i])
        assert np.array_equal(so[3], bo[3])
        single.free()


def test_query_async_in_cuda_graph(env):
    torch, pspc = env
    g, rank, pairs_fn = P.workload("rmat12_ef16")
    dev = torch.device("cuda:0")
    ix = pspc.Index.build(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                          torch.from_numpy(rank).to(dev))
    q = 50000
    pairs = torch.from_numpy(pairs_fn(q)).to(dev)
    d = torch.zeros(q, dtype=torch.uint16, device=dev)
    c = torch.zeros(q, dtype=torch.uint64, device=dev)
    f = torch.zeros(q, dtype=torch.uint8, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ix.query_async(pairs, d, c, f, err, stream=s)  # first call outside capture
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ix.query_async(pairs, d, c, f, err, stream=s)
    for trial in range(2):
        new = torch.from_numpy(pairs_fn(q) if trial == 0 else P.query_pairs(g.n, q, 123)).to(dev)
        pairs.copy_(new)
        d.zero_()
        c.zero_()
        graph.replay()
        torch.cuda.synchronize()
        rd, rc, rf = ix.query(new)
        assert np.array_equal(d.cpu().numpy(), rd.cpu().numpy())
        assert np.array_equal(c.cpu().numpy(), rc.cpu().numpy())
        assert np.array_equal(f.cpu().numpy(), rf.cpu().numpy())
        assert int(err.item()) == 0
    # an out-of-range id sets the device flag
    pairs[0, 1] = g.n
    graph.replay()
    torch.cuda.synchronize()
    assert int(err.item()) == 1


def test_autotuner_keeps_answers(env):
    torch, pspc = env
    from paper_2212_00977_gb300 import autotune

    autotune.clear()
    g, rank, pairs_fn = P.workload("rmat12_ef16")
    dev = torch.device("cuda:0")
    rp, col, rk = (torch.from_numpy(a).to(dev) for a in (g.row_ptr, g.col, rank))
    opts = autotune.tune_build(lambda **o: pspc.Index.build(g.n, rp, col, rk, **o), g.n, g.arcs)
    ix = pspc.Index.build(g.n, rp, col, rk, **opts)
    ref = oracle.OracleIndex(g, rank)
    off, hub, dist, cnt, ovf = ix.export()
    r = ref.export()
    assert np.array_equal(hub, r.hub) and np.array_equal(cnt, r.cnt)
    pairs = torch.from_numpy(pairs_fn(20000)).to(dev)
    choice = autotune.tune_query(ix, pairs)
    assert choice in autotune.QUERY_VARIANTS
    d, c, f = ix.query(pairs)
    rd, rc, rf, _ = ref.query(pairs.cpu().numpy())
    assert np.array_equal(d.cpu().numpy(), rd) and np.array_equal(c.cpu().numpy(), rc)


def test_every_graph_on_six_vertices_in_one_batch(env):
    """Exhaustive: all 2^15 graphs on 6 vertices, each under a seeded random
    order, built as one batch; every graph's labels equal the oracle's of
    that graph alone, and all its ordered pairs answer like the oracle."""
    torch, pspc = env
    n = 6
    pairs6 = [(a, b) for a in range(n) for b in range(a + 1, n)]
    rng = np.random.default_rng(6)
    graphs, ranks = [], []
    for mask in range(1 << len(pairs6)):
        e = np.array([pairs6[k] for k in range(len(pairs6)) if mask >> k & 1], np.int64).reshape(-1, 2)
        graphs.append(P.csr_from_edges(n, e))
        ranks.append(rng.permutation(n).astype(np.int32))
    ix = pspc.Index.build_batch([(g.n, g.row_ptr, g.col, r) for g, r in zip(graphs, ranks)])
    try:
        off, hub, dist, cnt, ovf = ix.export()
        allp = np.array([(a, b) for a in range(n) for b in range(n)], np.int32)
        d, c, f = ix.query(np.concatenate([allp + n * i for i in range(len(graphs))]).astype(np.int32))
        for i, (g, r) in enumerate(zip(graphs, ranks)):
            ref_ix = oracle.OracleIndex(g, r)
            ref = ref_ix.export()
            lo, hi = off[n * i], off[n * (i + 1)]
            assert np.array_equal(off[n * i:n * (i + 1) + 1] - lo, ref.off), i
            assert np.array_equal(hub[lo:hi] - n * i, ref.hub), i
            assert np.array_equal(dist[lo:hi], ref.dist) and np.array_equal(cnt[lo:hi], ref.cnt), i
            rd, rc, rf, _ = ref_ix.query(allp)
            s = slice(len(allp) * i, len(allp) * (i + 1))
            assert np.array_equal(d[s], rd) and np.array_equal(c[s], rc) and np.array_equal(f[s], rf), i
    finally:
        ix.free()
