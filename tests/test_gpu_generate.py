"""Device generators (pg_graph_generate): the seeded synthetic graphs drawn
and built on the GPU equal the host generators' CSR arc for arc (the same
counter-based draws, loops dropped, duplicates removed, rows sorted), and
propagations on them equal the oracle on the host graph."""
import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu


CASES = [
    ("er", dict(n=10_000, avg_degree=8), lambda: I.er(10_000, 8, 0), 0),
    ("er", dict(n=3_001, avg_degree=5.5), lambda: I.er(3_001, 5.5, 17), 17),
    ("rmat", dict(scale=12, edge_factor=16, directed=True), lambda: I.rmat(12, 16, 2, True), 2),
    ("rmat", dict(scale=13, edge_factor=8, directed=False), lambda: I.rmat(13, 8, 5, False), 5),
    ("grid", dict(rows=90, cols=70, p_delete=0.05), lambda: I.grid(90, 70, 0.05, 3), 3),
    ("grid", dict(rows=1, cols=50, p_delete=0.0), lambda: I.grid(1, 50, 0.0, 4), 4),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_device_generator_equals_host_generator(case):
    kind, kw, host, seed = CASES[case]
    g = host()
    G = pg.Graph.generate(kind, seed, relabel=False, **kw)
    assert (G.n, G.m) == (g.n, g.m)
    rp, col = G.csr()
    assert np.array_equal(rp, np.asarray(g.row_ptr))
    assert np.array_equal(col, np.asarray(g.col))


def test_generated_graph_propagates_like_the_host_graph():
    """A relabelled (by default) device-built R-MAT: counts and m_active
    equal the oracle's on the host-built graph."""
    g = I.rmat(17, 8, 31, directed=False)
    seeds = I.seeds(g.n, 200, 32)
    want = oracle.run(g, seeds)
    G = pg.Graph.generate("rmat", 31, scale=17, edge_factor=8, directed=False)
    assert G.relabelled and (G.n, G.m) == (g.n, g.m)
    res = pg.propagate_p(G, seeds)
    assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, want["m_active"])
    Gr = pg.Graph.generate("rmat", 2, scale=12, edge_factor=16, directed=True, reverse=True)
    gd = I.rmat(12, 16, 2, True)
    seeds2 = I.seeds(gd.n, 64, 3)
    rp, col = np.asarray(gd.row_ptr), np.asarray(gd.col)
    src = np.repeat(np.arange(gd.n, dtype=np.int32), np.diff(rp))
    wt = oracle.run(I.from_arcs(gd.n, src, col), seeds2)  # the transpose
    rr = pg.propagate_p(Gr, seeds2)
    assert rr.rounds == wt["rounds"] and np.array_equal(rr.counts, wt["counts"])


@pytest.mark.slow
def test_device_generator_scale_22():
    g = I.rmat(22, 16, 2, directed=True)
    G = pg.Graph.generate("rmat", 2, scale=22, edge_factor=16, directed=True, relabel=False)
    rp, col = G.csr()
    assert np.array_equal(rp, np.asarray(g.row_ptr)) and np.array_equal(col, np.asarray(g.col))
