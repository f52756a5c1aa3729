"""The input recipe is deterministic, and the oracle's shortest-path counts
agree with an independent library (networkx) on random graphs."""
from __future__ import annotations

import hashlib

import numpy as np
import pytest

import oracle
import pspc_inputs as P


def digest(g, rank=None):
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col) + ((rank,) if rank is not None else ()):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("name", ["ba2000", "rmat12_ef16", "grid32", "grid32@td", "ba2000@hybrid5"])
def test_workloads_are_deterministic(name):
    g1, r1, p1 = P.workload(name)
    g2, r2, p2 = P.workload(name)
    assert digest(g1, r1) == digest(g2, r2)
    assert np.array_equal(p1(1000), p2(1000))
    # symmetric CSR, ascending rows, no self-loops
    src = np.repeat(np.arange(g1.n), g1.degree())
    assert not np.any(src == g1.col)
    fwd = set(zip(src.tolist(), g1.col.tolist()))
    assert all((b, a) in fwd for a, b in fwd)
    for v in range(min(g1.n, 500)):
        row = g1.col[g1.row_ptr[v]:g1.row_ptr[v + 1]]
        assert np.all(np.diff(row) > 0)


def test_ba_batch_is_deterministic():
    a = P.ba_batch(count=6, n_range=(50, 300), m_range=(1, 4), seed=5)
    b = P.ba_batch(count=6, n_range=(50, 300), m_range=(1, 4), seed=5)
    for (n1, rp1, c1, r1), (n2, rp2, c2, r2) in zip(a, b):
        assert n1 == n2 and np.array_equal(rp1, rp2) and np.array_equal(c1, c2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("seed", range(3))
def test_oracle_counts_match_networkx(seed):
    nx = pytest.importorskip("networkx")
    g = P.barabasi_albert(120, 2, 40 + seed)
    rank = P.degree_rank(g, "random", seed)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(g.edges().tolist())
    rng = np.random.default_rng(seed)
    pairs = rng.integers(0, g.n, size=(60, 2)).astype(np.int32)
    d, c, f, _ = oracle.OracleIndex(g, rank).query(pairs)
    for (s, t), dd, cc in zip(pairs.tolist(), d.tolist(), c.tolist()):
        if s == t:
            assert (dd, cc) == (0, 1)
            continue
        paths = list(nx.all_shortest_paths(G, s, t))
        assert dd == len(paths[0]) - 1
        assert cc == len(paths)
