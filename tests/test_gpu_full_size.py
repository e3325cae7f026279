"""Full-size parity: the benchmark workload in the launch configuration
bench.py times (event-timed plain launches) and with the CUDA-graph loop,
the 4096 x 4096 grid (~8,000 rounds), and sampled seed columns of the
scale-26 undirected R-MAT (2.1 B arcs, relabelled internally by default).
Counts and m_active are integers and must match the oracle exactly; metrics
within 1e-12 relative."""
import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _same(res, want, mact=True):
    assert res.rounds == want["rounds"]
    bad = np.argwhere(res.counts != want["counts"])
    assert bad.size == 0, f"mismatch (round, seed): {bad[:5].tolist()}"
    if mact:
        assert np.array_equal(res.m_active, want["m_active"])


def _metrics_close(res, want, n):
    got = pg.metrics(res, n)
    for k in ("diameter", "eff_diameter", "R_last", "dist_sum"):
        assert got[k] == want[k], k
    for k in ("avg_distance", "avg_distance_incl_self", "connectivity_rate", "reachable_pairs",
              "eff_diameter_interp"):
        assert got[k] == pytest.approx(want[k], rel=1e-12, abs=0.0), k


def _passes_m_active(g, dmat, rounds, planes=64):
    """PROPAGATE-S's m_active: each pass's own (its seed block's distances),
    summed over the passes."""
    total = np.zeros(rounds + 2, dtype=np.uint64)
    for b in range(0, dmat.shape[1], planes):
        sub = np.ascontiguousarray(dmat[:, b:b + planes])
        part = oracle.m_active(g, sub, int(sub.max()) + 1)
        total[:part.size] += part
    return total


def test_benchmark_workload_rmat22_directed_s256():
    g = I.rmat(22, 16, 2, directed=True)
    seeds = I.seeds(g.n, 256, 2)
    want = oracle.run(g, seeds, with_distances=True)
    mact_s = _passes_m_active(g, want.pop("dmat"), want["rounds"])
    G = pg.Graph.from_inputs(g)
    res_timed = pg.propagate_p(G, seeds, opts=pg.options(timing=1))  # bench's timed region
    _same(res_timed, want)
    _metrics_close(res_timed, want["metrics"], g.n)
    _same(pg.propagate_p(G, seeds), want)  # CUDA-graph loop
    res_s = pg.propagate_s(G, seeds, opts=pg.options(timing=1))  # 4 passes as words
    _same(res_s, want, mact=False)
    assert np.array_equal(res_s.m_active, mact_s)  # each pass's own m_active, summed
    assert res_s.seed_edge_traversals > 0


def test_grid_4096_deleted_edges_s128():
    g = I.grid(4096, 4096, 0.05, 3)
    seeds = I.seeds(g.n, 128, 3)
    want = oracle.run(g, seeds, with_distances=True)
    mact_s = _passes_m_active(g, want.pop("dmat"), want["rounds"])
    assert want["rounds"] > 4000  # long-diameter regime
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, seeds)
    _same(res, want)
    _metrics_close(res, want["metrics"], g.n)
    res_s = pg.propagate_s(G, seeds)  # its 2 passes of 64 planes as 2 words
    _same(res_s, want, mact=False)
    assert np.array_equal(res_s.m_active, mact_s)


def _first_round_m_active(g, seeds):
    """m_active(1): every out-neighbour of a seed is revisited in round 1
    (none is saturated yet when the seeds are at least two), so the entry is
    the sum of their in-degrees. The graph is symmetric, so a seed's
    out-neighbours are its own row."""
    assert not g.directed and len(seeds) >= 2
    rp, col = np.asarray(g.row_ptr), np.asarray(g.col)
    nbrs = np.unique(np.concatenate([col[rp[x]:rp[x + 1]] for x in seeds]))
    return int((rp[nbrs + 1] - rp[nbrs]).sum())


def test_rmat26_undirected_s512_sampled_columns():
    g = I.rmat(26, 16, 2, directed=False)
    seeds = I.seeds(g.n, 512, 2)
    G = pg.Graph.from_inputs(g)
    assert G.relabelled  # a skewed graph: renumbered internally by default
    res = pg.propagate_p(G, seeds)
    deg = np.diff(g.row_ptr)
    live = [i for i in range(512) if deg[seeds[i]] > 0]
    pick = np.array(live[:6] + [i for i in (0, 511) if i not in live[:6]], dtype=np.int64)
    hist, _, dmat = oracle.seed_histograms(g, seeds[pick], threads=len(pick),
                                           with_distances=True)
    T = max(hist.shape[1] - 1, res.rounds)
    want = np.zeros((len(pick), T + 1), np.int64)
    want[:, :hist.shape[1]] = hist
    got = np.zeros_like(want)
    got[:, :res.rounds + 1] = res.counts[:, pick].T
    assert np.array_equal(got, want)
    assert res.rounds >= hist.shape[1] - 1
    # m_active of the 512-seed run: its first round by the definition
    assert int(res.m_active[1]) == _first_round_m_active(g, seeds)
    # the sampled seeds alone, at full size: counts and every m_active entry
    sub = pg.propagate_p(G, np.ascontiguousarray(seeds[pick]))
    mact = oracle.m_active(g, dmat, hist.shape[1], threads=16)
    assert sub.rounds == hist.shape[1] - 1
    assert np.array_equal(sub.counts.T, hist.astype(np.uint32))
    assert np.array_equal(sub.m_active, mact)
    res_s = pg.propagate_s(G, seeds)
    assert np.array_equal(res_s.counts, res.counts)
    # PROPAGATE-S: each 64-plane pass's own first round, summed
    assert int(res_s.m_active[1]) == sum(_first_round_m_active(g, seeds[b:b + 64])
                                         for b in range(0, 512, 64))
