"""Full-size parity on the large workloads, on outputs the oracle computes
one by one: whole hub columns (from the definition: two BFSs per hub), the
labels of sampled vertices restricted to the highest-ranked hubs (from the
oracle's hub-pushing build stopped after those hubs), and queries from
sampled sources against breadth-first path counting, overflow flags
included."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pspc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as lib

    lib.load()
    return lib


def _build(pspc, g, rank, **kw):
    import torch

    d = torch.device("cuda:0")
    return pspc.Index.build(g.n, torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col).to(d),
                            torch.from_numpy(rank).to(d), **kw)


def _check(ix, g, rank, hubs, verts, K, sources, n_pairs, seed):
    # hub columns
    for w in hubs:
        gd, gc, gf = ix.hub_column(int(w))
        od, oc, of = oracle.hub_column(g, rank, int(w))
        assert np.array_equal(gd, od), f"hub {w}: distances"
        assert np.array_equal(gc, oc) and np.array_equal(gf, of), f"hub {w}: counts"
    # labels of sampled vertices restricted to the K highest-ranked hubs
    part = oracle.OracleIndex(g, rank, max_hubs=K).export()
    off, hub, dist, cnt, ovf = ix.export_vertices(verts)
    for i, v in enumerate(verts):
        a, b = int(off[i]), int(off[i + 1])
        keep = rank[hub[a:b]] < K
        got = list(zip(hub[a:b][keep].tolist(), dist[a:b][keep].tolist(), cnt[a:b][keep].tolist(),
                       ovf[a:b][keep].tolist()))
        assert got == part.of(int(v)), f"vertex {v}"
        assert (np.diff(rank[hub[a:b]]) > 0).all() and hub[b - 1] == v and dist[b - 1] == 0
    # queries from sampled sources
    rng = np.random.default_rng(seed)
    pairs = np.stack([np.repeat(np.asarray(sources, np.int32), n_pairs // len(sources)),
                      rng.integers(0, g.n, n_pairs // len(sources) * len(sources)).astype(np.int32)], 1)
    d, c, f = ix.query(pairs)
    for s in sources:
        bd, bc, bf = oracle.bfs_count(g, int(s))
        sel = pairs[:, 0] == s
        t = pairs[sel, 1]
        assert np.array_equal(d[sel].astype(np.int32), np.where(bd[t] < 0, 0xFFFF, bd[t]))
        assert np.array_equal(c[sel], bc[t]) and np.array_equal(f[sel], bf[t])
    return f


def test_grid256_full_size(pspc):
    """256x256 grid, 10% of edges deleted, largest component, random ties:
    ~500 levels and counts beyond 2^64 (overflow flags)."""
    g, rank, _ = P.workload("grid256")
    ix = _build(pspc, g, rank)
    st = ix.stats()
    assert st["levels"] > 400 and st["overflow_entries"] > 0
    rng = np.random.default_rng(5)
    order = np.argsort(rank)
    hubs = list(order[:3]) + list(rng.choice(g.n, 5, replace=False))
    verts = rng.choice(g.n, 300, replace=False)
    f = _check(ix, g, rank, hubs, verts, K=64, sources=list(rng.choice(g.n, 6, replace=False)),
               n_pairs=60000, seed=6)
    assert f.any()  # long grid paths overflow 64 bits


def test_rmat20_full_size(pspc):
    """R-MAT scale 20, edge factor 8, random ties (2.5e9 label entries)."""
    g, rank, _ = P.workload("rmat20")
    ix = _build(pspc, g, rank)
    rng = np.random.default_rng(7)
    order = np.argsort(rank)
    hubs = list(order[:3]) + list(order[rng.choice(200000, 3, replace=False)])
    verts = order[rng.choice(g.n - 500000, 300, replace=False)]  # skip most isolated vertices
    _check(ix, g, rank, hubs, verts, K=12, sources=list(order[rng.choice(300000, 4, replace=False)]),
           n_pairs=40000, seed=8)
