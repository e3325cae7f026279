"""CUDA path vs the CPU oracle: every per-round, per-seed count bit-exact,
m_active exact, metrics within 1e-12 relative, PROPAGATE-P == PROPAGATE-S,
every schedule identical. Runs through the C ABI (ctypes binding)."""
import ctypes
import functools

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import _abi
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL = 1e-12  # derived FP64 metrics: both sides divide identical integer sums


def _oracle_p(g, seeds):
    return oracle.run(g, seeds)


def _oracle_s_mactive(g, seeds, planes, rounds):
    """m_active of PROPAGATE-S: the per-pass measure summed over passes."""
    _, _, dmat = oracle.seed_histograms(g, seeds, with_distances=True)
    total = np.zeros(rounds + 2, dtype=np.uint64)
    for b in range(0, len(seeds), planes):
        sub = np.ascontiguousarray(dmat[:, b:b + planes])
        ecc = sub.max()
        part = oracle.m_active(g, sub, int(ecc) + 1)
        total[:part.size] += part
    return total


def _assert_metrics(res, want, n):
    got = pg.metrics(res, n)
    for k in ("diameter", "eff_diameter", "R_last", "dist_sum"):
        assert got[k] == want[k], k
    for k in ("eff_diameter_interp", "avg_distance", "avg_distance_incl_self",
              "connectivity_rate", "reachable_pairs"):
        assert got[k] == pytest.approx(want[k], rel=REL, abs=0.0), k


def _assert_same(res, want, check_mactive=True):
    assert res.rounds == want["rounds"]
    assert res.counts.shape == want["counts"].shape
    bad = np.argwhere(res.counts != want["counts"])
    assert bad.size == 0, f"first mismatches (round, seed): {bad[:5].tolist()}"
    if check_mactive:
        assert np.array_equal(res.m_active, want["m_active"]), (res.m_active, want["m_active"])


@functools.lru_cache(maxsize=None)
def _cfg1():
    g = I.er(10_000, 8, 0)
    seeds = I.seeds(g.n, 64, 1)
    return g, seeds, _oracle_p(g, seeds)


# ---------------------------------------------------------------- config 1
def test_cfg1_er_propagate_p_default():
    g, seeds, want = _cfg1()
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, seeds)
    _assert_same(res, want)
    _assert_metrics(res, want["metrics"], g.n)


@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("test_changed", [1, 2])
@pytest.mark.parametrize("sparse_push", [1, 2])
def test_cfg1_every_schedule_identical(direction, lanes, test_changed, sparse_push):
    g, seeds, want = _cfg1()
    G = pg.Graph.from_inputs(g)
    o = pg.options(direction=direction, group_lanes=lanes, test_changed=test_changed,
                   sparse_push=sparse_push)
    _assert_same(pg.propagate_p(G, seeds, opts=o), want)


@pytest.mark.parametrize("graphs,timing", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_cfg1_launch_modes_identical(graphs, timing):
    g, seeds, want = _cfg1()
    G = pg.Graph.from_inputs(g)
    o = pg.options(use_graphs=graphs, timing=timing)
    for _ in range(2):  # second call reuses the cached workspace / graph
        _assert_same(pg.propagate_p(G, seeds, opts=o), want)
    st = G.last_stats()
    assert st["sweeps"] == want["rounds"] + 1
    assert st["m_active_total"] == int(want["m_active"].sum())
    if timing:
        assert st["ms_pull"] > 0 and st["pull_launches"] >= st["sweeps"]


@pytest.mark.parametrize("planes", [1, 5, 64])
def test_cfg1_propagate_s_equals_p_and_oracle(planes):
    g, seeds, want = _cfg1()
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_s(G, seeds, opts=pg.options(planes_per_pass=planes))
    _assert_same(res, want, check_mactive=False)
    assert np.array_equal(res.m_active, _oracle_s_mactive(g, seeds, planes, want["rounds"]))
    _assert_metrics(res, want["metrics"], g.n)


# ------------------------------------------------------ ragged seed counts
@pytest.mark.parametrize("s", [1, 2, 3, 63, 64, 65, 100, 130, 257, 513, 700])
def test_ragged_seed_counts(s):
    g = I.er(3001, 5, 11)
    seeds = I.seeds(g.n, s, 100 + s)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    _assert_same(pg.propagate_p(G, seeds), want)
    _assert_same(pg.propagate_s(G, seeds), want, check_mactive=False)


# ---------------------------------------------------- directed / skewed
@pytest.mark.parametrize("scale,ef,s", [(12, 8, 64), (13, 16, 256), (11, 4, 100)])
def test_directed_rmat(scale, ef, s):
    g = I.rmat(scale, ef, 7, directed=True)
    seeds = I.seeds(g.n, s, 5)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    for d in (pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
        for tc in (1, 2):
            o = pg.options(direction=d, test_changed=tc)
            _assert_same(pg.propagate_p(G, seeds, opts=o), want)
    res_s = pg.propagate_s(G, seeds)
    _assert_same(res_s, want, check_mactive=False)


@pytest.mark.parametrize("lanes", [1, 2, 8, 32])
def test_long_rows_split_into_pieces(lanes):
    # hubs of R-MAT and a star centre: rows far longer than a piece
    g = I.rmat(12, 16, 3, directed=False)
    seeds = I.seeds(g.n, 130, 9)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    for d in (pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
        o = pg.options(group_lanes=lanes, direction=d)
        _assert_same(pg.propagate_p(G, seeds, opts=o), want)
    st = I.star(5000)
    sd = np.array([0, 17, 4999], dtype=np.int32)
    want = _oracle_p(st, sd)
    S = pg.Graph.from_inputs(st)
    _assert_same(pg.propagate_p(S, sd, opts=pg.options(group_lanes=lanes)), want)


def test_grid_small_every_direction():
    g = I.grid(90, 70, 0.05, 3)
    seeds = I.seeds(g.n, 128, 4)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    for d in (pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
        _assert_same(pg.propagate_p(G, seeds, opts=pg.options(direction=d)), want)


# ------------------------------------------------------------ exact mode
@pytest.mark.parametrize("kind", ["er", "digraph", "grid"])
def test_exact_mode_all_nodes_seeds(kind):
    g = {"er": lambda: I.er(300, 3, 2), "digraph": lambda: I.random_digraph(250, 600, 3),
         "grid": lambda: I.grid(12, 17, 0.0, 0)}[kind]()
    seeds = np.arange(g.n, dtype=np.int32)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, seeds)
    _assert_same(res, want)
    _assert_metrics(res, want["metrics"], g.n)
    _assert_same(pg.propagate_s(G, seeds), want, check_mactive=False)
    if kind == "grid":
        m = pg.metrics(res, g.n)
        assert m["reachable_pairs"] == g.n * g.n and m["diameter"] == 12 + 17 - 2


# ------------------------------------------------------------ edge cases
def test_single_node_no_edges():
    g = I.from_arcs(1, np.array([], np.int32), np.array([], np.int32))
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, np.array([0], np.int32))
    assert res.rounds == 0 and res.counts.tolist() == [[1]]
    assert res.m_active.tolist() == [0, 0]
    assert pg.propagate_s(G, np.array([0], np.int32)).counts.tolist() == [[1]]


def test_isolated_nodes_and_unreachable():
    src = np.array([0, 1, 5], np.int32)
    dst = np.array([1, 2, 6], np.int32)
    g = I.from_arcs(9, src, dst)  # nodes 3, 4, 7, 8 isolated
    seeds = np.array([0, 3, 5, 8, 2], np.int32)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    _assert_same(pg.propagate_p(G, seeds), want)
    _assert_same(pg.propagate_s(G, seeds), want, check_mactive=False)


def test_long_path_moves_counts_window():
    g = I.path(1500)
    seeds = np.array([0, 700, 1499, 3], np.int32)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    for graphs in (0, 1):
        o = pg.options(window_rows=37, use_graphs=graphs)
        res = pg.propagate_p(G, seeds, opts=o)
        _assert_same(res, want)
    _assert_same(pg.propagate_s(G, seeds, opts=pg.options(window_rows=50)), want,
                 check_mactive=False)


def test_max_rounds_too_small_returns_erange_with_prefix():
    g = I.path(40)
    seeds = np.array([0], np.int32)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    L = _abi.lib()
    cap = 10
    counts = np.zeros((cap + 1, 1), np.uint32)
    mact = np.zeros(cap + 2, np.uint64)
    c = _abi.Counts(s=1, max_rounds=cap, rounds=0, reserved=0, counts=counts.ctypes.data,
                    m_active=mact.ctypes.data)
    rc = L.pg_propagate_p(G._h, np.array([0], np.int32).ctypes.data, 1, ctypes.byref(c),
                          None, None)
    assert rc == _abi.PG_ERANGE
    assert c.rounds == cap + 1
    assert np.array_equal(counts[:, 0], want["counts"][:cap + 1, 0])
    # the graph stays usable
    _assert_same(pg.propagate_p(G, seeds), want)


def test_invalid_seeds_rejected():
    g = I.er(100, 4, 1)
    G = pg.Graph.from_inputs(g)
    for bad in ([1, 1], [100], [-1], []):
        with pytest.raises(pg.PropagateError) as e:
            pg.propagate_p(G, np.array(bad, np.int32))
        assert e.value.status == _abi.PG_EINVAL
    _assert_same(pg.propagate_p(G, np.array([5, 7], np.int32)),
                 _oracle_p(g, np.array([5, 7], np.int32)))


@pytest.mark.parametrize("what", ["unsorted", "dup", "range", "rowptr", "last"])
def test_invalid_csr_rejected(what):
    rp = np.array([0, 2, 3, 5], np.int64)
    col = np.array([1, 2, 0, 0, 1], np.int32)
    if what == "unsorted":
        col[0], col[1] = 2, 1
    elif what == "dup":
        col[1] = 1
    elif what == "range":
        col[2] = 3
    elif what == "rowptr":
        rp[1] = 4
    else:
        rp[3] = 4
    with pytest.raises(pg.PropagateError) as e:
        pg.Graph.from_csr(rp, col, 3)
    assert e.value.status == _abi.PG_EINVAL


def _big_valid_csr(seed):
    """A larger CSR (rows of 0-40 arcs, many empty) whose columns strictly
    increase within each row and descend at most row starts."""
    rng = np.random.default_rng(seed)
    n = 5000
    deg = rng.integers(0, 41, n)
    deg[rng.random(n) < 0.2] = 0
    rows = [np.sort(rng.choice(n, int(d), replace=False)).astype(np.int32) for d in deg]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(deg)
    return rp, np.concatenate(rows), n


@pytest.mark.parametrize("pos", [0, 1, 2, 3, 4, 5, 6, 7])
def test_invalid_csr_descent_anywhere_in_a_row(pos):
    """The column check counts descents (col[j-1] >= col[j]) against the rows
    starting on one: a single swap inside any row, at any offset of the
    4-arc groups the check reads, is rejected; the unswapped CSR (descents
    only at row starts, empty rows between) is accepted."""
    rp, col, n = _big_valid_csr(61)
    G = pg.Graph.from_csr(rp, col, n)  # valid
    G.close()
    rows = [v for v in range(n) if rp[v + 1] - rp[v] >= 2]
    # a row whose second arc sits at the requested offset within a quad
    v = next(v for v in rows if (rp[v] + 1) % 8 == pos)
    bad = col.copy()
    bad[rp[v]], bad[rp[v] + 1] = bad[rp[v] + 1], bad[rp[v]]
    with pytest.raises(pg.PropagateError) as e:
        pg.Graph.from_csr(rp, bad, n)
    assert e.value.status == _abi.PG_EINVAL
    dup = col.copy()
    dup[rp[v] + 1] = dup[rp[v]]  # a repeated arc
    with pytest.raises(pg.PropagateError):
        pg.Graph.from_csr(rp, dup, n)


def test_pinned_host_csr_upload_is_exact():
    """A CSR in pinned host memory (the end-to-end leg's input): the device
    copy equals the input, with an arc count whose bytes are not a multiple
    of 16 and from a source 16-byte aligned or starting mid-buffer; counts
    equal those of the same graph uploaded from pageable memory."""
    torch = pytest.importorskip("torch")
    g = I.er(400_000, 48, 71)
    rp, col = np.array(g.row_ptr), np.array(g.col)
    drop = 1 + (int(col.size) % 4 == 1)  # leave m % 4 != 0
    rp = rp.copy()
    rp[-1] -= drop
    col = col[:col.size - drop]
    assert (col.size * 4) % 16 != 0 and col.size * 4 >= 64 << 20
    rp_p = torch.from_numpy(rp).pin_memory()
    big = torch.empty(col.size + 3, dtype=torch.int32).pin_memory()  # source at +12 bytes
    big[3:] = torch.from_numpy(col)
    col_p = big[3:]
    assert col_p.data_ptr() % 16 != 0
    big4 = torch.empty(col.size, dtype=torch.int32).pin_memory()
    big4.copy_(torch.from_numpy(col))
    seeds = I.seeds(g.n, 64, 72)
    want = pg.propagate_p(pg.Graph.from_csr(rp, col, g.n, directed=True), seeds)
    for c in (big4, col_p):
        G = pg.Graph.from_csr(rp_p.numpy(), c.numpy(), g.n, directed=True, relabel=False)
        r2, c2 = G.csr()
        assert np.array_equal(r2, rp) and np.array_equal(c2, col)
        res = pg.propagate_p(G, seeds)
        assert np.array_equal(res.counts, want.counts)
        G.close()


def test_device_pointer_graph_equals_host_graph():
    torch = pytest.importorskip("torch")
    g = I.rmat(12, 8, 21, directed=True)
    seeds = I.seeds(g.n, 96, 2)
    want = _oracle_p(g, seeds)
    rp = torch.from_numpy(np.array(g.row_ptr)).cuda()
    col = torch.from_numpy(np.array(g.col)).cuda()
    G = pg.Graph.from_csr(rp, col, g.n, directed=True)
    _assert_same(pg.propagate_p(G, seeds), want)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _assert_same(pg.propagate_p(G, seeds), want)


def test_repeated_calls_different_widths_reuse_graph():
    g = I.er(5000, 6, 8)
    G = pg.Graph.from_inputs(g)
    for s in (64, 512, 3, 256, 64):
        seeds = I.seeds(g.n, s, s)
        _assert_same(pg.propagate_p(G, seeds), _oracle_p(g, seeds))


# ------------------------------------------- the paper's literal direction
def _transpose(g):
    """Host transpose of a CSR over in-edges (the in-CSR of the reversed
    graph), with sorted rows."""
    n = g.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    src = np.asarray(g.col, dtype=np.int64)
    order = np.lexsort((rows, src))
    col_t = rows[order].astype(np.int32)
    rp_t = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp_t, src + 1, 1)
    return I.Graph(n=n, row_ptr=np.cumsum(rp_t), col=col_t, directed=True, name=g.name + "_T",
                   meta={})


@pytest.mark.parametrize("fn", ["p", "s"])
def test_reverse_flag_counts_backward_balls(fn):
    """PG_REVERSE: counts of nodes that reach each seed, i.e. the forward
    balls of the reversed graph (the oracle on the explicit transpose)."""
    g = I.rmat(12, 8, 91, directed=True)
    seeds = I.seeds(g.n, 100, 92)
    want = oracle.run(_transpose(g), seeds)
    G = pg.Graph.from_inputs(g, reverse=True)
    res = (pg.propagate_p if fn == "p" else pg.propagate_s)(G, seeds)
    assert res.rounds == want["rounds"]
    assert np.array_equal(res.counts, want["counts"])
    fwd = oracle.run(g, seeds)
    assert not np.array_equal(fwd["counts"][:2], want["counts"][:2])  # the direction matters


def test_graph_create_free_cycles():
    """Graphs created and freed over and over (the end-to-end pattern), two
    shapes alternating: every result stays exact."""
    g1 = I.rmat(12, 8, 141, directed=True)
    g2 = I.grid(50, 50, 0.05, 142)
    s1 = I.seeds(g1.n, 300, 143)
    s2 = I.seeds(g2.n, 100, 144)
    w1, w2 = oracle.run(g1, s1), oracle.run(g2, s2)
    for k in range(6):
        for g, sd, w in ((g1, s1, w1), (g2, s2, w2)):
            G = pg.Graph.from_inputs(g)
            r = pg.propagate_p(G, sd)
            rs = pg.propagate_s(G, sd)
            assert r.rounds == w["rounds"] and np.array_equal(r.counts, w["counts"])
            assert np.array_equal(rs.counts, w["counts"])
            G.close()


# ------------------------------------------------------------- relabelling
@functools.lru_cache(maxsize=None)
def _relabel_cases():
    return [
        (I.rmat(12, 8, 151, directed=True), 130, 152),
        (I.rmat(13, 16, 153, directed=False), 512, 154),
        (I.star(5000), 65, 155),
        (I.grid(90, 70, 0.05, 156), 64, 157),
        (I.er(3000, 6, 158), 257, 159),
        (I.path(1500), 3, 160),
    ]


@pytest.mark.parametrize("case", range(6))
def test_relabel_gives_identical_counts(case):
    """PG_RELABEL renumbers the nodes internally (hubs first); seeds go in and
    counts come out in the caller's ids and order, so counts, m_active and
    metrics equal the oracle's on the graph as given, for P, S and every
    direction."""
    g, s, sd = _relabel_cases()[case]
    seeds = I.seeds(g.n, s, sd)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g, relabel=True)
    assert G.relabelled
    for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
        res = pg.propagate_p(G, seeds, opts=pg.options(direction=direction))
        _assert_same(res, want)
    _assert_metrics(res, want["metrics"], g.n)
    res_s = pg.propagate_s(G, seeds)
    assert res_s.rounds == want["rounds"] and np.array_equal(res_s.counts, want["counts"])
    assert np.array_equal(res_s.m_active,
                          _oracle_s_mactive(g, seeds, 64, want["rounds"])[:res_s.m_active.size])


def test_relabel_with_reverse_and_graph_copies():
    """A relabelled directed graph pulled over its transpose (PG_REVERSE), and
    PROPAGATE-S passes run over copies of a relabelled graph (each copy's
    seeds mapped through the same permutation)."""
    g = I.rmat(12, 8, 91, directed=True)
    seeds = I.seeds(g.n, 100, 92)
    want = oracle.run(_transpose(g), seeds)
    G = pg.Graph.from_inputs(g, reverse=True, relabel=True)
    res = pg.propagate_p(G, seeds)
    assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])
    g2 = I.rmat(11, 8, 161, directed=False)
    s2 = I.seeds(g2.n, 200, 162)
    want2 = _oracle_p(g2, s2)
    G2 = pg.Graph.from_inputs(g2, relabel=True)
    r2 = pg.propagate_s(G2, s2, opts=pg.options(planes_per_pass=16, passes_together=4))
    assert r2.rounds == want2["rounds"] and np.array_equal(r2.counts, want2["counts"])


def test_relabel_default_follows_the_degree_skew():
    """By default a large skewed graph (R-MAT) is relabelled and a lattice is
    not; PG_KEEP_ORDER turns it off; the counts are the same either way."""
    g = I.rmat(17, 8, 171, directed=False)
    seeds = I.seeds(g.n, 128, 172)
    G = pg.Graph.from_inputs(g)
    K = pg.Graph.from_inputs(g, relabel=False)
    assert G.relabelled and not K.relabelled
    a, b = pg.propagate_p(G, seeds), pg.propagate_p(K, seeds)
    assert a.rounds == b.rounds and np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.m_active, b.m_active)
    h, _ = oracle.seed_histograms(g, seeds[:8])
    assert np.array_equal(a.counts[:h.shape[1], :8].T, h.astype(np.uint32))
    assert not a.counts[h.shape[1]:, :8].any()
    grid = I.grid(400, 300, 0.05, 173)
    assert not pg.Graph.from_inputs(grid).relabelled


def _active_rows_from_distances(g, seeds):
    """|A_t| per round from the oracle's BFS distances: rows with a zero bit
    before round t and an in-neighbour at distance t-1 from some seed (the
    rows whose in-degrees m_active sums)."""
    hist, _, dmat = oracle.seed_histograms(g, seeds, with_distances=True)
    T = hist.shape[1] - 1
    rp, col = np.asarray(g.row_ptr), np.asarray(g.col)
    deg = np.diff(rp)
    rows = np.repeat(np.arange(g.n), deg)
    out = np.zeros(T + 2, dtype=np.int64)
    for t in range(1, T + 2):
        changed = (dmat == t - 1).any(axis=1)
        unsat = ((dmat > t - 1) | (dmat < 0)).any(axis=1)
        hit = np.zeros(g.n, dtype=bool)
        hit[rows[changed[col]]] = True
        out[t] = int((hit & unsat).sum())
    return out


@pytest.mark.parametrize("which", ["er", "rmat_directed", "grid"])
def test_active_rows_match_distances(which):
    """pg_stats.active_rows (the |A_t| of the per-round byte count) equals the
    count restated from the oracle's distances, in every direction."""
    if which == "er":
        g, seeds = _cfg1()[0], _cfg1()[1]
    elif which == "rmat_directed":
        g = I.rmat(12, 8, 181, directed=True)
        seeds = I.seeds(g.n, 130, 182)
    else:
        g = I.grid(60, 50, 0.05, 183)
        seeds = I.seeds(g.n, 64, 184)
    want = int(_active_rows_from_distances(g, seeds).sum())
    G = pg.Graph.from_inputs(g)
    for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
        pg.propagate_p(G, seeds, opts=pg.options(direction=direction))
        assert G.last_stats()["active_rows"] == want, direction


# --------------------------------------------------- TMA-gathered dense rounds
@pytest.mark.parametrize("s", [512, 256, 130])
@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE])
def test_tma_gather_dense_rounds_match_the_oracle(s, direction):
    """tma_gather = 2: the dense rounds copy the neighbours' delta rows into
    shared memory with tile::gather4 (rows of 8 or 4 words); counts, m_active
    and active rows equal the oracle's, for PROPAGATE-P and for PROPAGATE-S
    with its passes as words, over rows cut into pieces (R-MAT hubs), with the
    captured round loop and with plain event-timed launches."""
    g = I.rmat(13, 16, 191, directed=False)
    seeds = I.seeds(g.n, s, 192)
    want = _oracle_p(g, seeds)
    G = pg.Graph.from_inputs(g)
    base = dict(direction=direction, tma_gather=2)
    for extra in (dict(), dict(timing=1), dict(test_changed=2), dict(test_changed=1)):
        res = pg.propagate_p(G, seeds, opts=pg.options(**base, **extra))
        assert G.last_stats()["dense_tma"] == 1
        _assert_same(res, want)
    if direction == pg.PG_DIR_DENSE:
        assert G.last_stats()["dense_tma"] == 1
        assert G.last_stats()["active_rows"] == int(_active_rows_from_distances(g, seeds).sum())
    res_s = pg.propagate_s(G, seeds, opts=pg.options(**base))
    assert res_s.rounds == want["rounds"] and np.array_equal(res_s.counts, want["counts"])
    assert np.array_equal(res_s.m_active,
                          _oracle_s_mactive(g, seeds, 64, want["rounds"])[:res_s.m_active.size])


def test_tma_gather_directed_and_reverse():
    """TMA-gathered dense rounds on a directed graph, forward and with
    PG_REVERSE (the pull over the out-edge transpose)."""
    g = I.rmat(12, 16, 193, directed=True)
    seeds = I.seeds(g.n, 300, 194)
    o = pg.options(direction=pg.PG_DIR_DENSE, tma_gather=2)
    _assert_same(pg.propagate_p(pg.Graph.from_inputs(g), seeds, opts=o), _oracle_p(g, seeds))
    want = oracle.run(_transpose(g), seeds)
    res = pg.propagate_p(pg.Graph.from_inputs(g, reverse=True), seeds, opts=o)
    assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])


# ------------------------------------------------ arc arrays in host memory
@pytest.mark.parametrize("which", ["rmat_directed", "rmat_undirected", "grid"])
def test_host_csr_counts_match_the_oracle(which):
    """PG_HOST_CSR keeps the arc arrays (columns, transpose, sliced-ELL copy)
    in pinned host memory, read by the kernels over the CPU-GPU link: the
    counts, m_active and metrics are the oracle's, in every direction, for
    P and S, relabelled or not, and over the transpose (PG_REVERSE)."""
    if which == "rmat_directed":
        g, s = I.rmat(12, 16, 201, directed=True), 200
    elif which == "rmat_undirected":
        g, s = I.rmat(13, 16, 202, directed=False), 512
    else:
        g, s = I.grid(80, 90, 0.05, 203), 128
    seeds = I.seeds(g.n, s, 204)
    want = _oracle_p(g, seeds)
    for relabel in (False, True):
        G = pg.Graph.from_inputs(g, host_csr=True, relabel=relabel)
        for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE):
            _assert_same(pg.propagate_p(G, seeds, opts=pg.options(direction=direction)), want)
        res_s = pg.propagate_s(G, seeds)
        assert res_s.rounds == want["rounds"] and np.array_equal(res_s.counts, want["counts"])
        G.close()
    if g.directed:
        wr = oracle.run(_transpose(g), seeds)
        r = pg.propagate_p(pg.Graph.from_inputs(g, host_csr=True, reverse=True), seeds)
        assert r.rounds == wr["rounds"] and np.array_equal(r.counts, wr["counts"])


def test_debug_bounds_build_gives_the_oracles_counts():
    """The PG_DEBUG_BOUNDS build, in a process of its own
    (PG_LIBRARY_VARIANT=debug-bounds): no gather is out of range on valid
    inputs (a bad index would make the call return PG_EDEVICE), and the
    counts equal the oracle's, for the per-lane, wide-row and TMA pulls."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, oracle, paper_2301_06499_gb300 as pg\n"
        "from paper_2301_06499_gb300 import inputs as I, _abi\n"
        "assert 'debug_bounds' in _abi.lib()._name\n"
        "cases = [(I.rmat(12, 16, 211, directed=True), 200, {}),\n"
        "         (I.rmat(13, 16, 212, directed=False), 512, {'tma_gather': 2}),\n"
        "         (I.grid(60, 70, 0.05, 213), 64, {}), (I.er(2000, 6, 214), 700, {})]\n"
        "for g, s, o in cases:\n"
        "    seeds = I.seeds(g.n, s, 215)\n"
        "    want = oracle.run(g, seeds)\n"
        "    G = pg.Graph.from_inputs(g)\n"
        "    for fn in (pg.propagate_p, pg.propagate_s):\n"
        "        r = fn(G, seeds, opts=pg.options(**o))\n"
        "        assert r.rounds == want['rounds'] and np.array_equal(r.counts, want['counts'])\n"
        "print('debug-bounds ok')\n")
    env = dict(os.environ, PG_LIBRARY_VARIANT="debug-bounds")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                         text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    assert "debug-bounds ok" in out.stdout


# ------------------------------------------------------------ push rounds
@pytest.mark.parametrize("case", ["er", "grid", "rmat_directed", "star", "path"])
def test_push_rounds_match_the_oracle(case):
    """sparse_push = 2: sparse rounds OR each changed row's delta into its
    out-neighbours with atomics (claims counted on the way); counts, m_active
    and active rows equal the oracle's in every direction, for PROPAGATE-P
    and PROPAGATE-S one pass at a time, with captured and plain launches."""
    if case == "er":
        g, seeds = _cfg1()[0], _cfg1()[1]
    elif case == "grid":
        g = I.grid(90, 70, 0.05, 221)
        seeds = I.seeds(g.n, 128, 222)
    elif case == "rmat_directed":
        g = I.rmat(12, 16, 223, directed=True)
        seeds = I.seeds(g.n, 256, 224)
    elif case == "star":
        g = I.star(5000)
        seeds = I.seeds(g.n, 65, 225)
    else:
        g = I.path(1500)
        seeds = np.array([0, 700, 1499], np.int32)
    want = _oracle_p(g, seeds)
    rows = int(_active_rows_from_distances(g, seeds).sum())
    G = pg.Graph.from_inputs(g)
    for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_SPARSE):
        for extra in (dict(), dict(timing=1), dict(test_changed=1), dict(group_lanes=4)):
            res = pg.propagate_p(G, seeds, opts=pg.options(direction=direction, sparse_push=2,
                                                           **extra))
            _assert_same(res, want)
            assert G.last_stats()["active_rows"] == rows
    one = pg.options(sparse_push=2, pass_words=1, passes_together=1, direction=pg.PG_DIR_SPARSE)
    res_s = pg.propagate_s(G, seeds, opts=one)
    assert res_s.rounds == want["rounds"] and np.array_equal(res_s.counts, want["counts"])
    assert np.array_equal(res_s.m_active,
                          _oracle_s_mactive(g, seeds, 64, want["rounds"])[:res_s.m_active.size])


@pytest.mark.parametrize("s", [300, 512])
def test_push_rounds_eight_words(s):
    """sparse_push = 2 on rows of 8 words (s = 300 and 512): the push runs
    in k_push, a kernel of its own launched after the pull; counts, m_active
    and active rows equal the oracle's, with captured and plain launches and
    with every round forced sparse."""
    for g, sd in ((I.grid(70, 60, 0.05, 231), 232), (I.rmat(12, 8, 233, directed=False), 234)):
        seeds = I.seeds(g.n, s, sd)
        want = _oracle_p(g, seeds)
        rows = int(_active_rows_from_distances(g, seeds).sum())
        G = pg.Graph.from_inputs(g)
        for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_SPARSE):
            for extra in (dict(), dict(use_graphs=0), dict(timing=1), dict(test_changed=1)):
                res = pg.propagate_p(G, seeds, opts=pg.options(direction=direction,
                                                               sparse_push=2, **extra))
                _assert_same(res, want)
                st = G.last_stats()
                assert st["active_rows"] == rows
                # zero, seed and post(0), then the pull, the push and the post
                # kernel in rounds 1..T+1 (the host loop may run idle rounds)
                full = 3 + 3 * (want["rounds"] + 1)
                if extra.get("use_graphs", 1) and not extra.get("timing", 0):
                    assert st["launches"] == full, (st["launches"], full)
                else:
                    assert st["launches"] >= full and (st["launches"] - 3) % 3 == 0
        G.close()


def test_push_rounds_reverse_and_relabelled():
    """Push rounds over the transpose (PG_REVERSE) of a relabelled digraph."""
    g = I.rmat(12, 8, 226, directed=True)
    seeds = I.seeds(g.n, 100, 227)
    want = oracle.run(_transpose(g), seeds)
    G = pg.Graph.from_inputs(g, reverse=True, relabel=True)
    res = pg.propagate_p(G, seeds, opts=pg.options(sparse_push=2, direction=pg.PG_DIR_SPARSE))
    assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, want["m_active"])
