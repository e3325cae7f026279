"""The allocation-free entry point (pg_propagate_p_noalloc) against the oracle
and against pg_propagate_p.

Some callers cannot allocate device memory once they run (a serving process
that reserves its memory up front, a loop that cannot take an allocation's
synchronisation); pg_propagate_p_noalloc serves them from a fixed device array
and must give exactly the counts of the allocating entry point, which are the
oracle's BFS distance histograms. Two calls in a row check that the shared
array's leftovers from one call never leak into the next. This file sorts
last so that a run stopping at the first failure has already run every other
test."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import _abi
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(lib, rp, col, n, m, seeds, max_rounds, stream):
    import torch
    s = int(seeds.size)
    counts = torch.full(((max_rounds + 1) * s,), 7, dtype=torch.int32, device="cuda")
    rounds = ctypes.c_int32(-1)
    rc = lib.pg_propagate_p_noalloc(rp.data_ptr(), col.data_ptr(), n, m, seeds.ctypes.data, s,
                                    counts.data_ptr(), max_rounds, ctypes.byref(rounds), stream)
    torch.cuda.synchronize()
    return rc, int(rounds.value), counts.cpu().numpy().view(np.uint32).reshape(max_rounds + 1, s)


def _device_csr(g):
    import torch
    rp = torch.from_numpy(np.array(g.row_ptr)).cuda()
    col = torch.from_numpy(np.array(g.col) if g.m else np.zeros(1, np.int32)).cuda()
    return rp, col


def test_noalloc_equals_propagate_p_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    lib = _abi.lib()
    g = I.er(10_000, 8, 0)
    rp, col = _device_csr(g)
    G = pg.Graph.from_csr(rp, col, g.n, directed=False)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    max_rounds = 64
    for s, seed in ((64, 1), (100, 5)):
        seeds = I.seeds(g.n, s, seed)
        want = pg.propagate_p(G, seeds)
        ref = oracle.run(g, seeds, with_m_active=False)
        rc, T, counts = _noalloc(lib, rp, col, g.n, g.m, seeds, max_rounds, stream)
        assert rc == _abi.PG_OK
        assert T == want.rounds == ref["rounds"]
        assert np.array_equal(counts[:T + 1], want.counts)  # integer counts: exact
        assert np.array_equal(counts[:T + 1], ref["counts"])
        assert not counts[T + 1:].any()


def test_noalloc_directed_rmat_matches_oracle():
    torch = pytest.importorskip("torch")
    lib = _abi.lib()
    g = I.rmat(12, 8, 21, directed=True)
    rp, col = _device_csr(g)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for s, seed in ((130, 3), (7, 4)):  # ragged last word, and one partial word
        seeds = I.seeds(g.n, s, seed)
        ref = oracle.run(g, seeds, with_m_active=False)
        rc, T, counts = _noalloc(lib, rp, col, g.n, g.m, seeds, 40, stream)
        assert rc == _abi.PG_OK
        assert T == ref["rounds"]
        assert np.array_equal(counts[:T + 1], ref["counts"])


def test_noalloc_erange_writes_the_prefix():
    pytest.importorskip("torch")
    lib = _abi.lib()
    g = I.path(40)
    rp, col = _device_csr(g)
    seeds = np.array([0], np.int32)
    ref = oracle.run(g, seeds, with_m_active=False)
    cap = 10
    rc, T, counts = _noalloc(lib, rp, col, g.n, g.m, seeds, cap, None)
    assert rc == _abi.PG_ERANGE
    assert T == cap + 1
    assert np.array_equal(counts[:, 0], ref["counts"][:cap + 1, 0])


@pytest.mark.parametrize("what", ["range", "rowptr"])
def test_noalloc_rejects_a_malformed_csr_on_the_device(what):
    torch = pytest.importorskip("torch")
    lib = _abi.lib()
    rp = np.array([0, 2, 3, 5], np.int64)
    col = np.array([1, 2, 0, 0, 1], np.int32)
    if what == "range":
        col[2] = 3  # a column index >= n
    else:
        rp[1] = 4  # row_ptr not monotone
    rp_d = torch.from_numpy(rp).cuda()
    col_d = torch.from_numpy(col).cuda()
    rc, _, _ = _noalloc(lib, rp_d, col_d, 3, 5, np.array([0], np.int32), 4, None)
    assert rc == _abi.PG_EINVAL
    # the entry point stays usable after a rejected call
    g = I.er(500, 6, 2)
    rp2, col2 = _device_csr(g)
    seeds = I.seeds(g.n, 33, 9)
    ref = oracle.run(g, seeds, with_m_active=False)
    rc, T, counts = _noalloc(lib, rp2, col2, g.n, g.m, seeds, 30, None)
    assert rc == _abi.PG_OK and T == ref["rounds"]
    assert np.array_equal(counts[:T + 1], ref["counts"])


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib = _abi.lib()
    n = _abi.PG_NOALLOC_SCRATCH_BYTES // 8  # 4 n words cannot fit
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    seeds = np.array([0, 1], np.int32)
    rc, _, _ = _noalloc(lib, rp, col, n, 0, seeds, 4, None)
    assert rc == _abi.PG_ETOOBIG
    assert b"fixed scratch" in lib.pg_strerror(rc)
