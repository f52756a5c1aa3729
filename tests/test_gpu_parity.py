"""GPU parity: the CUDA index and query answers equal the CPU oracle bit for
bit (tolerance zero: every value is an integer). All calls go through the C
ABI via the Python binding."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle
import pspc_inputs as P
from tests import _graphs as G

pytestmark = pytest.mark.gpu

M64 = 1 << 64


@pytest.fixture(scope="module")
def pspc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as lib

    lib.load()
    return lib


def gpu_index(pspc, g, rank, device=True, **kw):
    import torch

    if device:
        d = torch.device("cuda:0")
        return pspc.Index.build(g.n, torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col).to(d),
                                torch.from_numpy(np.ascontiguousarray(rank, np.int32)).to(d), **kw)
    return pspc.Index.from_graph(g, rank, **kw)


def assert_index_equal(ix, ref):
    off, hub, dist, cnt, ovf = ix.export()
    assert np.array_equal(off, ref.off), "label sizes differ"
    assert np.array_equal(hub, ref.hub), "hubs differ"
    assert np.array_equal(dist, ref.dist), "distances differ"
    assert np.array_equal(cnt, ref.cnt), "counts differ"
    assert np.array_equal(ovf, ref.ovf), "overflow flags differ"


def gpu_query(ix, pairs, device=True):
    import torch

    if device:
        d, c, f = ix.query(torch.from_numpy(pairs).cuda())
        return d.cpu().numpy(), c.cpu().numpy(), f.cpu().numpy()
    return ix.query(pairs)


# --- the paper's example ---

def test_paper_table(pspc):
    g, rank, table, (s, t, sd, c) = G.load_paper_table()
    ix = gpu_index(pspc, g, rank)
    off, hub, dist, cnt, ovf = ix.export()
    for v in range(10):
        got = [(int(hub[i]), int(dist[i]), int(cnt[i])) for i in range(off[v], off[v + 1])]
        assert got == table[v], v
    d, cc, f = gpu_query(ix, np.array([[s, t], [t, s]], np.int32))
    assert d.tolist() == [sd, sd] and cc.tolist() == [c, c] and f.tolist() == [0, 0]


# --- small graphs against the oracle, across table capacities ---

CAPS = [dict(), dict(cand_capacity=1024, label_capacity=1024), dict(map_kind=2, label_capacity=1024),
        dict(map_kind=3), dict(landmarks=-1), dict(landmarks=64, map_kind=3), dict(paradigm=1),
        dict(paradigm=1, map_kind=3, cand_capacity=1024)]


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("caps", range(len(CAPS)))
def test_random_graphs_index_and_all_pairs(pspc, seed, caps):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 120))
    g = G.gnp(n, float(rng.choice([0.03, 0.08, 0.2])), 300 + seed)
    rank = G.random_rank(n, seed) if seed % 2 else G.degree_rank(g)
    ref_ix = oracle.OracleIndex(g, rank)
    ix = gpu_index(pspc, g, rank, **CAPS[caps])
    assert_index_equal(ix, ref_ix.export())
    pairs = np.array(list(itertools.product(range(n), range(n))), np.int32)
    d, c, f = gpu_query(ix, pairs)
    rd, rc, rf, _ = ref_ix.query(pairs)
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)


@pytest.mark.parametrize("case", range(len(G.closed_forms())))
def test_closed_forms(pspc, case):
    g, s, t, sd, cnt = G.closed_forms()[case]
    for rank in (G.degree_rank(g), G.random_rank(g.n, case)):
        ix = gpu_index(pspc, g, rank)
        assert_index_equal(ix, oracle.OracleIndex(g, rank).export())
        d, c, f = gpu_query(ix, np.array([[s, t], [t, s], [s, s]], np.int32))
        assert d.tolist() == [sd, sd, 0]
        assert c.tolist() == [cnt % M64, cnt % M64, 1]
        assert f.tolist() == [int(cnt >= M64)] * 2 + [0]


@pytest.mark.parametrize("k", [63, 64, 65])
def test_diamond_chain_label_overflow(pspc, k):
    g = G.diamond_chain(k)
    rank = np.arange(g.n, dtype=np.int32)
    ix = gpu_index(pspc, g, rank)
    ref = oracle.OracleIndex(g, rank).export()
    assert_index_equal(ix, ref)
    assert ix.stats()["overflow_entries"] == int(ref.ovf.sum())
    assert (int(ref.ovf.sum()) > 0) == (k >= 64)


def test_offchip_counts_carry_past_2_64(pspc):
    """500 hubs over a width-2 ladder 66 layers deep: every ladder vertex
    pulls 1000 entries for 500 hubs, more than an on-chip table of 1024 slots
    holds, so with cand_capacity=1024 the level runs off chip; at layer 65
    each hub's count is 2^63 + 2^63 (a carry past 2^64 in the split sums),
    at 66 the pulled entries already carry the flag. The index equals the
    oracle's with every map kind and in the default configuration."""
    g = G.hub_ladder(500, 66)
    rank = np.arange(g.n, dtype=np.int32)
    ref = oracle.OracleIndex(g, rank).export()
    assert ref.ovf.sum() > 0
    for kw in (dict(), dict(cand_capacity=1024), dict(cand_capacity=1024, map_kind=2, label_capacity=1024),
               dict(cand_capacity=1024, map_kind=3), dict(cand_capacity=1024, paradigm=1)):
        ix = gpu_index(pspc, g, rank, **kw)
        assert_index_equal(ix, ref)
        if kw:
            assert sum(l["offchip_vertices"] for l in ix.level_stats()) >= 2 * 60, kw
        ix.free()


def test_trees_isolated_components_and_tiny(pspc):
    for g, rank in [
        (G.random_tree(300, 1), G.random_rank(300, 1)),
        (P.csr_from_edges(7, np.array([(0, 1), (1, 2), (4, 5)])), np.array([3, 0, 4, 6, 1, 5, 2], np.int32)),
        (P.csr_from_edges(1, np.zeros((0, 2), np.int64)), np.array([0], np.int32)),
        (P.csr_from_edges(5, np.zeros((0, 2), np.int64)), np.array([4, 3, 2, 1, 0], np.int32)),
        (G.path(2), np.array([1, 0], np.int32)),
    ]:
        ref = oracle.OracleIndex(g, rank)
        ix = gpu_index(pspc, g, rank)
        assert_index_equal(ix, ref.export())
        pairs = np.array(list(itertools.product(range(g.n), range(g.n))), np.int32).reshape(-1, 2)
        d, c, f = gpu_query(ix, pairs)
        rd, rc, rf, _ = ref.query(pairs)
        assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)


# --- the named workloads that the oracle builds in seconds ---

@pytest.mark.parametrize("name", ["ba2000", "rmat12_ef16", "grid32", "grid64"])
def test_workload_full_index(pspc, name):
    g, rank, pairs_fn = P.workload(name)
    ref = oracle.OracleIndex(g, rank)
    ix = gpu_index(pspc, g, rank)
    assert_index_equal(ix, ref.export())
    pairs = pairs_fn(200000)
    d, c, f = gpu_query(ix, pairs)
    rd, rc, rf, _ = ref.query(pairs)
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)


def test_ba2000_all_pairs_vs_bfs(pspc):
    """Barabasi-Albert n=2,000, m=4: every ordered pair against BFS counting."""
    g, rank, _ = P.workload("ba2000")
    ix = gpu_index(pspc, g, rank)
    n = g.n
    pairs = np.stack([np.repeat(np.arange(n, dtype=np.int32), n), np.tile(np.arange(n, dtype=np.int32), n)], 1)
    d, c, f = gpu_query(ix, pairs)
    d = d.reshape(n, n)
    c = c.reshape(n, n)
    for s in range(n):
        bd, bc, bf = oracle.bfs_count(g, s)
        assert np.array_equal(d[s].astype(np.int32), np.where(bd < 0, 0xFFFF, bd)), s
        assert np.array_equal(c[s], bc), s
    assert not f.any()


# --- invariance: capacities, host vs device buffers, repeated builds ---

def test_layout_invariance(pspc):
    g, rank, pairs_fn = P.workload("rmat12_ef16")
    ref = oracle.OracleIndex(g, rank).export()
    pairs = pairs_fn(50000)
    outs = []
    for kw, dev in [(dict(), True), (dict(), False), (dict(cand_capacity=1024, label_capacity=1024), True),
                    (dict(cand_capacity=8192, label_capacity=16384), True), (dict(arena_entries=1), True),
                    (dict(map_kind=2), True), (dict(map_kind=3), True), (dict(map_kind=2, label_capacity=1024), True),
                    (dict(granular=True), True), (dict(max_ctas=8), True),
                    (dict(granular=True, cand_capacity=1024, label_capacity=1024, map_kind=2), True)]:
        ix = gpu_index(pspc, g, rank, device=dev, **kw)
        assert_index_equal(ix, ref)
        outs.append(gpu_query(ix, pairs, device=dev))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


# --- bad inputs are rejected with PSPC_E_INVAL ---

def test_invalid_inputs(pspc):
    g = G.cycle(6)
    rank = np.arange(6, dtype=np.int32)
    bad = []
    bad.append((6, g.row_ptr, g.col, np.array([0, 1, 2, 3, 4, 4], np.int32)))  # not a permutation
    bad.append((6, g.row_ptr, g.col, np.array([0, 1, 2, 3, 4, 6], np.int32)))  # out of range
    col = g.col.copy()
    col[0] = 0  # self loop at vertex 0
    bad.append((6, g.row_ptr, col, rank))
    col = g.col.copy()
    col[0], col[1] = col[1], col[0]  # unsorted row
    bad.append((6, g.row_ptr, col, rank))
    asym_rp = np.array([0, 1, 3, 5], np.int64)
    asym_col = np.array([1, 0, 2, 1, 0], np.int32)  # 2->0 without 0->2
    bad.append((3, asym_rp, asym_col, np.arange(3, dtype=np.int32)))
    rp = g.row_ptr.copy()
    rp[2], rp[3] = rp[3], rp[2]  # row_ptr not monotone
    bad.append((6, rp, g.col, rank))
    for n, rp_, col_, rk in bad:
        with pytest.raises(pspc.PSPCError) as ei:
            pspc.Index.build(n, rp_, col_, rk)
        assert ei.value.code == pspc.PSPC_E_INVAL
    ix = gpu_index(pspc, g, rank)
    with pytest.raises(pspc.PSPCError) as ei:
        ix.query(np.array([[0, 6]], np.int32))
    assert ei.value.code == pspc.PSPC_E_INVAL
    d, c, f = ix.query(np.zeros((0, 2), np.int32))
    assert len(d) == 0
    # on-chip tables larger than the device's shared memory are rejected
    with pytest.raises(pspc.PSPCError) as ei:
        pspc.Index.build(6, g.row_ptr, g.col, rank, cand_capacity=16384, label_capacity=16384)
    assert ei.value.code == pspc.PSPC_E_INVAL


# --- full-size workloads: every entry, and queries, against the definition ---

def test_rmat16_full_size(pspc):
    """R-MAT scale 16, edge factor 16 (65,536 vertices, 45M label entries):
    every entry of the index against the definition, hub column by hub
    column for all 65,536 hubs (the entry total equals the index size, so
    no label holds anything else), labels in strict hub-rank order with the
    self entry last, and 10^6 query pairs against breadth-first counting
    (one search per distinct source, all sources)."""
    g, rank, pairs_fn = P.workload("rmat16")
    ix = gpu_index(pspc, g, rank)
    off, hub, dist, cnt, ovf = ix.export()
    _check_whole_index(g, rank, off, hub, dist, cnt, ovf)
    pairs = pairs_fn(1_000_000)
    d, c, f = gpu_query(ix, pairs)
    od, oc, of, _ = oracle.spc_pairs(g, pairs)
    assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
    assert ix.stats()["entries"] == len(hub)


def test_rmat16_small_tables_routing(pspc):
    """R-MAT scale 16 with on-chip candidate tables of 1,024 slots: most
    heavy vertices of levels 2-4 overflow them, so whole size classes are
    routed to the off-chip pass without an attempt; every entry of the
    index against the definition, as with the default tables."""
    g, rank, pairs_fn = P.workload("rmat16")
    ix = gpu_index(pspc, g, rank, cand_capacity=1024)
    ls = ix.level_stats()
    assert sum(l["routed_vertices"] for l in ls) > 1000
    assert all(l["routed_vertices"] <= l["offchip_vertices"] for l in ls)
    off, hub, dist, cnt, ovf = ix.export()
    _check_whole_index(g, rank, off, hub, dist, cnt, ovf)
    ix.free()


def test_long_labels_few_levels(pspc):
    """K(2, 8500) with the middle ranked first: three levels, and the two
    outer vertices hold labels of 8,501 entries, more than the finalize
    keeps on chip by default (they are merged again with a larger buffer);
    every entry against the definition, labels in strict hub order."""
    m = 8500
    g = G.bipartite_2m(m)
    rank = np.arange(g.n, dtype=np.int32)
    ix = gpu_index(pspc, g, rank)
    assert ix.label_sizes([m, m + 1]).min() == m + 1
    off, hub, dist, cnt, ovf = ix.export()
    _check_whole_index(g, rank, off, hub, dist, cnt, ovf)
    ix.free()


def _check_whole_index(g, rank, off, hub, dist, cnt, ovf):
    """Every entry of an exported index equals the definition (all hub
    columns), and labels are strictly increasing in hub rank and end with
    the vertex itself at distance 0."""
    n = g.n
    assert off[0] == 0 and off[-1] == len(hub) and (np.diff(off) >= 1).all()
    r = rank[hub].astype(np.int64)
    owner = np.repeat(np.arange(n), np.diff(off))
    same = owner[1:] == owner[:-1]
    assert (r[1:][same] > r[:-1][same]).all()
    last = off[1:] - 1
    assert np.array_equal(hub[last], np.arange(n)) and (dist[last] == 0).all() and (cnt[last] == 1).all()
    assert (r <= rank[owner]).all()
    bad, ent, first = oracle.check_columns(g, rank, np.arange(n), off, hub, dist, cnt, ovf)
    assert bad == 0, first
    assert ent == len(hub)


def test_query_group_invariance(pspc):
    """Answers do not depend on how many lanes merge-join one pair."""
    for name in ("ba2000", "grid32"):
        g, rank, pairs_fn = P.workload(name)
        ref = oracle.OracleIndex(g, rank)
        ix = gpu_index(pspc, g, rank)
        pairs = pairs_fn(100000)
        rd, rc, rf, _ = ref.query(pairs)
        for lanes in (8, 16, 32, 64, 128, 256, pspc.PSPC_QUERY_BY_SOURCE, pspc.PSPC_QUERY_BY_SOURCE_HASH, 0):
            ix.set_query_group(lanes)
            d, c, f = gpu_query(ix, pairs)
            assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
        with pytest.raises(pspc.PSPCError):
            ix.set_query_group(12)


def test_query_variants_long_labels(pspc):
    """Labels many chunks long (grid 128: hundreds to thousands of entries,
    many hubs tied at the minimum): every query variant, including the
    by-source position table and hash, equals breadth-first path counting. Runs of 100 pairs per source and uniform pairs."""
    g, rank, pairs_fn = P.workload("grid128")
    rng = np.random.default_rng(5)
    src = rng.integers(0, g.n, 300)
    runs = np.stack([np.repeat(src, 100), rng.integers(0, g.n, 30000)], axis=1)
    pairs = np.concatenate([runs, pairs_fn(20000)]).astype(np.int32)
    pairs = pairs[rng.permutation(len(pairs))]
    rd, rc, rf, _ = oracle.spc_pairs(g, pairs)
    ix = gpu_index(pspc, g, rank)
    sizes = ix.label_sizes()
    assert sizes.max() > 1000 and sizes.mean() > 256
    for lanes in (pspc.PSPC_QUERY_BY_SOURCE, pspc.PSPC_QUERY_BY_SOURCE_HASH, 256, 128, 64, 32, 8, 0):
        ix.set_query_group(lanes)
        d, c, f = gpu_query(ix, pairs)
        assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
    ix.free()


def test_by_source_many_tied_hubs(pspc):
    """K(2, m) with the middle ranked first: L(s) and L(t) share m hubs, all
    at distance sum 2, so one pair has m matches tied at the minimum (more
    than a warp's on-chip list of them holds); every variant returns (2, m)
    for (s, t) and (2, 2) between middle vertices, as the oracle does."""
    m = 700
    g = G.bipartite_2m(m)
    rank = np.arange(g.n, dtype=np.int32)
    rng = np.random.default_rng(2)
    st = np.tile(np.array([[m, m + 1], [m + 1, m]], np.int32), (3000, 1))
    mid = rng.integers(0, m, (4000, 2)).astype(np.int32)
    pairs = np.concatenate([st, mid])
    pairs = pairs[rng.permutation(len(pairs))]
    rd, rc, rf, _ = oracle.OracleIndex(g, rank).query(pairs)
    assert rd[(pairs[:, 0] == m) & (pairs[:, 1] == m + 1)].tolist() == [2] * 3000
    assert set(rc[(pairs[:, 0] == m) & (pairs[:, 1] == m + 1)].tolist()) == {m}
    ix = gpu_index(pspc, g, rank)
    assert ix.label_sizes([m, m + 1]).min() >= m
    for lanes in (pspc.PSPC_QUERY_BY_SOURCE, pspc.PSPC_QUERY_BY_SOURCE_HASH, 256, 8, 0):
        ix.set_query_group(lanes)
        d, c, f = gpu_query(ix, pairs)
        assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
    ix.free()


def test_by_source_skew_repeats_and_overflow(pspc):
    """The by-source query path (pairs sorted by source, L(s) on chip):
    one source holding thousands of pairs (runs cut across many items),
    s = t pairs, every pair of a small graph many times over, and counts
    that overflow 2^64; answers equal the oracle's and every other variant's."""
    rng = np.random.default_rng(11)
    g, rank, pairs_fn = P.workload("ba2000")
    cases = []
    hot = np.stack([np.full(5000, 7), rng.integers(0, g.n, 5000)], axis=1)
    same = np.repeat(rng.integers(0, g.n, 3000)[:, None], 2, axis=1)
    cases.append((g, rank, np.concatenate([hot, same, pairs_fn(20000)]).astype(np.int32)))
    dg = G.diamond_chain(65)
    drank = np.arange(dg.n, dtype=np.int32)
    allp = np.array([(s, t) for s in range(dg.n) for t in range(dg.n)], np.int32)
    cases.append((dg, drank, np.concatenate([allp] * 3)))
    for gg, rk, pairs in cases:
        pairs = pairs[rng.permutation(len(pairs))]
        rd, rc, rf, _ = oracle.OracleIndex(gg, rk).query(pairs)
        ix = gpu_index(pspc, gg, rk)
        for lanes in (pspc.PSPC_QUERY_BY_SOURCE, pspc.PSPC_QUERY_BY_SOURCE_HASH, 256, 8):
            ix.set_query_group(lanes)
            d, c, f = gpu_query(ix, pairs)
            assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
            d, c, f = gpu_query(ix, pairs, device=False)
            assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
        if gg is dg:
            assert rf.any()
        for lanes in (pspc.PSPC_QUERY_BY_SOURCE, pspc.PSPC_QUERY_BY_SOURCE_HASH, 0):
            ix.set_query_group(lanes)
            for bad_pair in ((gg.n, 0), (-1, 3), (3, gg.n), (7, -5)):
                bad = pairs.copy()
                bad[len(bad) // 2] = bad_pair
                with pytest.raises(pspc.PSPCError) as e:
                    gpu_query(ix, bad)
                assert e.value.code == 1, (lanes, bad_pair)
            d, c, f = gpu_query(ix, pairs)  # the index still answers
            assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf), lanes
        ix.free()


@pytest.mark.parametrize("map_kind", [1, 2, 3])
def test_grid64_every_map_kind(pspc, map_kind):
    """Many levels and overflowing counts, under each way of testing label
    membership."""
    g, rank, pairs_fn = P.workload("grid64")
    ref = oracle.OracleIndex(g, rank)
    ix = gpu_index(pspc, g, rank, map_kind=map_kind)
    assert_index_equal(ix, ref.export())


def test_export_vertices_and_hub_column(pspc):
    g, rank, _ = P.workload("ba2000")
    ix = gpu_index(pspc, g, rank)
    ref = oracle.OracleIndex(g, rank).export()
    verts = np.array([5, 0, 1999, 17, 5], np.int32)
    off, hub, dist, cnt, ovf = ix.export_vertices(verts)
    for i, v in enumerate(verts):
        got = [(int(hub[j]), int(dist[j]), int(cnt[j]), int(ovf[j])) for j in range(off[i], off[i + 1])]
        assert got == ref.of(int(v))
    for w in (0, 3, 1999):
        d, c, f = ix.hub_column(w)
        od, oc, of = oracle.hub_column(g, rank, w)
        assert np.array_equal(d, od) and np.array_equal(c, oc) and np.array_equal(f, of)
    with pytest.raises(pspc.PSPCError):
        ix.export_vertices(np.array([2000], np.int32))
    with pytest.raises(pspc.PSPCError):
        ix.hub_column(-1)


@pytest.mark.parametrize("name", ["grid64@td", "grid64@hybrid5", "ba2000@hybrid5", "rmat12_ef16@td"])
def test_order_variants_full_index(pspc, name):
    """The hybrid and tree-decomposition orders (Section "Vertex Order")
    give other indexes; each equals the oracle's under the same order."""
    g, rank, pairs_fn = P.workload(name)
    ref = oracle.OracleIndex(g, rank)
    ix = gpu_index(pspc, g, rank)
    assert_index_equal(ix, ref.export())
    pairs = pairs_fn(20000)
    rd, rc, rf, _ = ref.query(pairs)
    d, c, f = gpu_query(ix, pairs)
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
    ix.free()


def _level_counts_from_oracle(g, rank):
    """Per level d >= 2, from the oracle's index and the graph alone: the
    pulled entries of rule 1 (for every arc u->v, the entries (h, d-1, c) of
    L(v) with h ranked above u) and the entries at distance d."""
    lab = oracle.OracleIndex(g, rank).export()
    n = g.n
    rank = np.asarray(rank, np.int64)
    owner = np.repeat(np.arange(n), np.diff(lab.off))
    orank = rank[owner]
    hrank = rank[lab.hub.astype(np.int64)]
    dist = (lab.dist & 0x7FFF).astype(np.int64)
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    ur, vr = rank[src], rank[g.col.astype(np.int64)]
    out = {}
    for d in range(2, int(dist.max()) + 2):
        keys = np.sort(orank[dist == d - 1] * n + hrank[dist == d - 1])
        raw = int((np.searchsorted(keys, vr * n + ur) - np.searchsorted(keys, vr * n)).sum())
        out[d] = (raw, int((dist == d).sum()))
    return out


@pytest.mark.parametrize("name", ["ba2000", "rmat12_ef16", "grid32"])
def test_level_counters_match_independent_count(pspc, name):
    """The per-level counters that the roofline's algorithmic bytes come
    from (pulled entries under rule 1, appended entries) equal a count made
    from the oracle's index, with the dense-prefix skip and the landmark
    filter on."""
    g, rank, _ = P.workload(name)
    want = _level_counts_from_oracle(g, rank)
    ix = gpu_index(pspc, g, rank)
    ls = ix.level_stats()
    for d, (raw, ent) in want.items():
        if d - 1 < len(ls):
            got = ls[d - 1]
            assert (got["raw_candidates"], got["entries"]) == (raw, ent), d
        else:
            assert raw == 0 and ent == 0, d
    ix.free()


@pytest.mark.parametrize("name", ["ba2000", "rmat12_ef16", "grid64", "grid32@td"])
def test_push_paradigm_full_index(pspc, name):
    """Algorithm PUSH (entries sent to per-vertex buckets, then merged)
    builds the same index as the pull: the oracle's, bit for bit."""
    g, rank, pairs_fn = P.workload(name)
    ref = oracle.OracleIndex(g, rank)
    ix = gpu_index(pspc, g, rank, paradigm=1)
    assert_index_equal(ix, ref.export())
    pairs = pairs_fn(20000)
    rd, rc, rf, _ = ref.query(pairs)
    d, c, f = gpu_query(ix, pairs)
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
    ix.free()
    with pytest.raises(pspc.PSPCError):
        gpu_index(pspc, g, rank, paradigm=2)
