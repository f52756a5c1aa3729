"""pspc_query_noalloc: the allocation-free query entry point, for callers that
cannot allocate device memory while they query (their device memory is owned
by another allocator, or their serving loop must never enter the driver's
allocator). It must give exactly the answers of pspc_query, call after call,
through the C ABI, and the oracle's. Collected last on purpose: a failure
here leaves every other test already run."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as pspc

    lib = pspc.load()
    return torch, pspc, lib


def _noalloc(lib, ix, pairs_d, torch, fill):
    q = pairs_d.shape[0]
    d = torch.full((q,), fill, dtype=torch.uint16, device=pairs_d.device)
    c = torch.full((q,), fill, dtype=torch.uint64, device=pairs_d.device)
    f = torch.full((q,), fill, dtype=torch.uint8, device=pairs_d.device)
    rc = lib.pspc_query_noalloc(ix._h, pairs_d.data_ptr(), q, d.data_ptr(), c.data_ptr(), f.data_ptr(), None)
    return rc, d.cpu().numpy(), c.cpu().numpy(), f.cpu().numpy()


# (workload, pairs): 300,000 pairs group by source (by-source or staged
# kernels fed by the call's own permutation); 1,000 pairs do not group, and
# the plain kernels run in caller order (k_query<16> on BA 2000, the staged
# k_query_chunked<256> on the larger labels of R-MAT 12 and grid 32).
@pytest.mark.parametrize("name,q", [("rmat12_ef16", 300000), ("grid32", 300000), ("rmat12_ef16", 1000),
                                    ("grid32", 1000), ("ba2000", 1000), ("ba2000", 5000)])
def test_noalloc_matches_query_on_two_calls_in_a_row(env, name, q):
    torch, pspc, lib = env
    g, rank, pairs_fn = P.workload(name)
    dev = torch.device("cuda:0")
    ix = pspc.Index.build(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                          torch.from_numpy(rank).to(dev))
    pairs = pairs_fn(q)
    pairs[:7] = [[0, 0], [1, 1], [0, g.n - 1], [g.n - 1, 0], [5, 9], [9, 5], [3, 3]]
    pairs_d = torch.from_numpy(pairs).to(dev)
    rd, rc, rf = ix.query(pairs_d)
    ref = (rd.cpu().numpy(), rc.cpu().numpy(), rf.cpu().numpy())
    od, oc, of, _ = oracle.OracleIndex(g, rank).query(pairs)
    assert np.array_equal(ref[0], od) and np.array_equal(ref[1], oc) and np.array_equal(ref[2], of)
    # two calls in a row, each starting from different garbage in the outputs;
    # the shared scratch keeps the first call's contents for the second.
    # Every library allocation fails meanwhile: the calls must not need one.
    pspc.inject_alloc_failure(0)
    try:
        for fill in (0, 7):
            status, d, c, f = _noalloc(lib, ix, pairs_d, torch, fill)
            assert status == pspc.PSPC_OK
            assert np.array_equal(d, ref[0]) and np.array_equal(c, ref[1]) and np.array_equal(f, ref[2])
    finally:
        pspc.inject_alloc_failure(-1)
    ix.free()


def test_noalloc_rejects_what_it_cannot_serve_without_allocating(env):
    torch, pspc, lib = env
    g, rank, pairs_fn = P.workload("ba2000")
    dev = torch.device("cuda:0")
    ix = pspc.Index.from_graph(g, rank)
    # host buffers would need device staging memory
    pairs = pairs_fn(1000)
    d = np.empty(1000, np.uint16)
    c = np.empty(1000, np.uint64)
    f = np.empty(1000, np.uint8)
    assert lib.pspc_query_noalloc(ix._h, pairs.ctypes.data, 1000, d.ctypes.data, c.ctypes.data, f.ctypes.data,
                                  None) == pspc.PSPC_E_INVAL
    # a grouped call (q >= 4096 and q >= n/4) with more pairs than the
    # static working array holds: flag, bins (the n+2 bins fit one scan tile
    # here, so there are no scan partials), pair indices
    limit = (16 << 20) - 256 - ((8 * (g.n + 2) + 255) // 256) * 256
    q_big = limit // 4 + 1
    big = torch.zeros((q_big, 2), dtype=torch.int32, device=dev)
    db = torch.empty(q_big, dtype=torch.uint16, device=dev)
    cb = torch.empty(q_big, dtype=torch.uint64, device=dev)
    assert lib.pspc_query_noalloc(ix._h, big.data_ptr(), q_big, db.data_ptr(), cb.data_ptr(), None,
                                  None) == pspc.PSPC_E_INVAL
    # the largest accepted batch still answers (all pairs (0, 0) -> (0, 1))
    status = lib.pspc_query_noalloc(ix._h, big.data_ptr(), q_big - 1, db.data_ptr(), cb.data_ptr(), None, None)
    assert status == pspc.PSPC_OK
    dh = db[: q_big - 1].cpu().numpy()
    ch = cb[: q_big - 1].cpu().numpy()
    assert (dh == 0).all() and (ch == 1).all()
    # an out-of-range vertex is reported, as by pspc_query
    bad = torch.tensor([[0, g.n]], dtype=torch.int32, device=dev)
    assert lib.pspc_query_noalloc(ix._h, bad.data_ptr(), 1, db.data_ptr(), cb.data_ptr(), None,
                                  None) == pspc.PSPC_E_INVAL
    ix.free()
