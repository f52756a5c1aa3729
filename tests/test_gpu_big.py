"""Full-size parity on the two large workloads (R-MAT scale 20, and the
256x256 grid with 10% of its edges deleted), against the definition, with
the oracle run in parallel on the host cores:

* the grid: every entry of the index, hub column by hub column for all
  hubs (the entry total equals the index size), and 10^6 query pairs
  against breadth-first counting;
* R-MAT 20 (2.5e9 entries, too many to export): whole hub columns for
  the 1,000 highest-ranked hubs and 3,000 random others, the labels of
  300 sampled vertices restricted to the 12 highest-ranked hubs, and
  10^5 query pairs (1,000 from each of 100 sources) against breadth-first
  counting.
Overflow flags are compared like every other field."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P
from tests.test_gpu_parity import _check_whole_index

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


def _check_queries(ix, g, pairs):
    import torch

    d, c, f = ix.query(torch.from_numpy(pairs).cuda())
    d, c, f = d.cpu().numpy(), c.cpu().numpy(), f.cpu().numpy()
    od, oc, of, _ = oracle.spc_pairs(g, pairs)
    assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
    return f


def test_grid256_full_size(pspc):
    """256x256 grid, 10% of edges deleted, largest component, random ties:
    ~500 levels and counts beyond 2^64 (overflow flags); every entry."""
    g, rank, pairs_fn = P.workload("grid256")
    ix = _build(pspc, g, rank)
    st = ix.stats()
    assert st["levels"] > 400 and st["overflow_entries"] > 0
    off, hub, dist, cnt, ovf = ix.export()
    _check_whole_index(g, rank, off, hub, dist, cnt, ovf)
    del off, hub, dist, cnt, ovf
    f = _check_queries(ix, g, pairs_fn(1_000_000))
    assert f.any()  # long grid paths overflow 64 bits
    ix.free()


def test_rmat20_full_size(pspc):
    """R-MAT scale 20, edge factor 8, random ties (2.5e9 label entries)."""
    g, rank, pairs_fn = P.workload("rmat20")
    ix = _build(pspc, g, rank)
    rng = np.random.default_rng(7)
    order = np.argsort(rank)
    hubs = np.concatenate([order[:1000], order[1000 + rng.choice(g.n - 1000, 3000, replace=False)]])
    for b in range(0, len(hubs), 250):
        batch = hubs[b:b + 250]
        od, oc, of = oracle.hub_columns(g, rank, batch)
        for i, w in enumerate(batch):
            gd, gc, gf = ix.hub_column(int(w))
            assert np.array_equal(gd, od[i]), f"hub {w}: distances"
            assert np.array_equal(gc, oc[i]) and np.array_equal(gf, of[i]), f"hub {w}: counts"
    # labels of sampled vertices restricted to the 12 highest-ranked hubs,
    # against the oracle's hub-pushing build stopped after those hubs
    K = 12
    part = oracle.OracleIndex(g, rank, max_hubs=K).export()
    verts = order[rng.choice(g.n - 500000, 300, replace=False)]  # skip most isolated vertices
    off, hub, dist, cnt, ovf = ix.export_vertices(verts)
    for i, v in enumerate(verts):
        a, b = int(off[i]), int(off[i + 1])
        keep = rank[hub[a:b]] < K
        got = list(zip(hub[a:b][keep].tolist(), dist[a:b][keep].tolist(), cnt[a:b][keep].tolist(),
                       ovf[a:b][keep].tolist()))
        assert got == part.of(int(v)), f"vertex {v}"
        assert (np.diff(rank[hub[a:b]]) > 0).all() and hub[b - 1] == v and dist[b - 1] == 0
    # queries: 1,000 pairs from each of 100 sources
    srcs = rng.choice(g.n, 100, replace=False).astype(np.int32)
    pairs = np.stack([np.repeat(srcs, 1000), rng.integers(0, g.n, 100_000).astype(np.int32)], 1)
    _check_queries(ix, g, pairs)
    ix.free()
