"""Host-side failure paths of the C ABI, on the GPU but without a GPU fault:
the distance limit (PSPC_E_DIST) at a caller's max_levels and at the 15-bit
storage limit of 32767, and allocation failures injected on the host
(PSPC_E_NOMEM, or PSPC_E_CUDA for another CUDA error) at every device
allocation of a build and of a query. After each failure the library keeps
working and its results still equal the oracle. With PSPC_E_INVAL (tested
with the bad inputs of the parity tests) every status the header declares
is reached."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P
from tests import _graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pspc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as lib

    lib.load()
    yield lib
    lib.inject_alloc_failure(-1)


def _same_index(ix, g, rank):
    got = ix.export()
    ref = oracle.OracleIndex(g, rank).export()
    for a, b in zip(got, (ref.off, ref.hub, ref.dist, ref.cnt, ref.ovf)):
        assert np.array_equal(a, b)


def test_max_levels_is_a_distance_limit(pspc):
    """The build succeeds when every label distance is within max_levels and
    fails with PSPC_E_DIST, returning no index, when one is beyond it."""
    g, rank, _ = P.workload("grid32")
    full = pspc.Index.from_graph(g, rank)
    top = full.stats()["levels"] - 1  # largest label distance
    full.free()
    ix = pspc.Index.from_graph(g, rank, max_levels=top)
    assert ix.stats()["levels"] == top + 1
    _same_index(ix, g, rank)
    ix.free()
    with pytest.raises(pspc.PSPCError) as e:
        pspc.Index.from_graph(g, rank, max_levels=top - 1)
    assert e.value.code == pspc.PSPC_E_DIST
    with pytest.raises(pspc.PSPCError) as e:
        pspc.Index.from_graph(g, rank, max_levels=1)
    assert e.value.code == pspc.PSPC_E_DIST


def _centroid_path_rank(n: int) -> np.ndarray:
    """Path 0 - 1 - ... - n-1 with vertex 0 ranked highest and the rest in
    centroid order (the middle of every remaining run next), so that labels
    stay small while hub 0 reaches the far end at distance n-1."""
    order = [0]
    runs = [(1, n - 1)]
    while runs:
        nxt = []
        for a, b in runs:
            if a > b:
                continue
            m = (a + b) // 2
            order.append(m)
            nxt += [(a, m - 1), (m + 1, b)]
        runs = nxt
    rank = np.empty(n, np.int32)
    rank[np.array(order)] = np.arange(n, dtype=np.int32)
    return rank


def test_distance_storage_limit_32767(pspc):
    """Distances are stored in 15 bits: a label distance of 32767 builds (and
    equals the oracle), one of 32768 is PSPC_E_DIST on the GPU, and the
    oracle refuses the same graph."""
    n = 32768
    g = G.path(n)
    rank = _centroid_path_rank(n)
    ix = pspc.Index.from_graph(g, rank)
    assert ix.stats()["levels"] == n
    _same_index(ix, g, rank)
    d, c, f = ix.query(np.array([[0, n - 1], [n - 1, 0], [1, n - 1]], np.int32))
    assert d.tolist() == [n - 1, n - 1, n - 2] and c.tolist() == [1, 1, 1]
    ix.free()
    g2 = G.path(n + 1)
    rank2 = _centroid_path_rank(n + 1)
    with pytest.raises(pspc.PSPCError) as e:
        pspc.Index.from_graph(g2, rank2)
    assert e.value.code == pspc.PSPC_E_DIST
    with pytest.raises(MemoryError):
        oracle.OracleIndex(g2, rank2)


@pytest.mark.parametrize("name,kw,status", [("ba2000", {}, "NOMEM"), ("grid32", {"map_kind": 2}, "NOMEM"),
                                            ("rmat12_ef16", {"paradigm": 1}, "NOMEM"), ("grid32", {}, "CUDA")])
def test_failure_at_every_allocation_of_a_build(pspc, name, kw, status):
    """Allocation k of a build fails, for every k, as out of memory or as
    another CUDA error: the build reports that status (PSPC_E_NOMEM or
    PSPC_E_CUDA) and returns no index; with no failure it succeeds, and the
    index equals the oracle's."""
    g, rank, _ = P.workload(name)
    code = pspc.PSPC_E_NOMEM if status == "NOMEM" else pspc.PSPC_E_CUDA
    k = 0
    while True:
        pspc.inject_alloc_failure(k, code)
        try:
            ix = pspc.Index.from_graph(g, rank, **kw)
        except pspc.PSPCError as e:
            assert e.code == code, (k, e)
            k += 1
            assert k < 2000
            continue
        finally:
            pspc.inject_alloc_failure(-1)
        break
    assert k > 5  # the build does allocate, and each failure point was reached
    _same_index(ix, g, rank)
    ix.free()


def test_out_of_memory_in_queries_and_exports(pspc):
    """With every allocation failing, pspc_query (host and device buffers)
    and pspc_export report PSPC_E_NOMEM; pspc_query_noalloc still answers.
    Afterwards every call works again and equals the oracle."""
    import torch

    g, rank, pairs_fn = P.workload("ba2000")
    ix = pspc.Index.from_graph(g, rank)
    pairs = pairs_fn(5000)
    rd, rc, rf, _ = oracle.OracleIndex(g, rank).query(pairs)
    dev = torch.device("cuda:0")
    pd = torch.from_numpy(pairs).to(dev)
    od = torch.empty(len(pairs), dtype=torch.uint16, device=dev)
    oc = torch.empty(len(pairs), dtype=torch.uint64, device=dev)
    of = torch.empty(len(pairs), dtype=torch.uint8, device=dev)
    lib = pspc.load()
    pspc.inject_alloc_failure(0)
    try:
        for p in (pairs, pd):
            with pytest.raises(pspc.PSPCError) as e:
                ix.query(p)
            assert e.value.code == pspc.PSPC_E_NOMEM
        with pytest.raises(pspc.PSPCError) as e:
            ix.export_vertices([0, 1])
        assert e.value.code == pspc.PSPC_E_NOMEM
        st = lib.pspc_query_noalloc(ix._h, pd.data_ptr(), len(pairs), od.data_ptr(), oc.data_ptr(),
                                    of.data_ptr(), None)
        assert st == pspc.PSPC_OK
    finally:
        pspc.inject_alloc_failure(-1)
    assert np.array_equal(od.cpu().numpy(), rd) and np.array_equal(oc.cpu().numpy(), rc)
    assert np.array_equal(of.cpu().numpy(), rf)
    d, c, f = ix.query(pairs)
    assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
    ix.free()
