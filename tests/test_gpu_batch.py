"""Batched PROPAGATE-P (pg_batch_*): every graph's per-round, per-seed counts
and its own m_active in a batch are bit-exact with the oracle and with the
same graph run alone through pg_propagate_p; the batch is credited exactly
the work of the plain runs (the work measure is defined by the method, not
the schedule)."""
import functools

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _mix():
    # sizes log-uniform in [500, 20000], every generator and width class
    return I.mix(24, 500, 20_000, 4)


def _width_class(s):
    w = (s + 63) // 64
    return w if w <= 2 else 4 if w <= 4 else -(-w // 8) * 8


def _plain(item):
    G = pg.Graph.from_inputs(item.graph)
    res = pg.propagate_p(G, item.seeds)
    st = G.last_stats()
    G.close()
    return res, st["seed_edge_traversals"]


def test_mix_covers_every_width_class():
    widths = {(it.s + 63) // 64 for it in _mix()}
    assert {1, 2}.issubset(widths) and any(w > 2 for w in widths)
    kinds = {it.graph.name.split("_")[0].rstrip("du") for it in _mix()}
    assert len(kinds) == 3, kinds


def test_batch_equals_plain_and_oracle():
    items = _mix()
    with pg.Batch() as b:
        idx = [b.add_inputs(it.graph, it.seeds) for it in items]
        b.run()
        st = b.stats()
        plain_work = 0
        for k, it in zip(idx, items):
            got = b.result(k)
            want, work = _plain(it)
            plain_work += work
            assert got.rounds == want.rounds, (it.graph.name, got.rounds, want.rounds)
            assert np.array_equal(got.counts, want.counts), it.graph.name
            assert np.array_equal(got.m_active, want.m_active), it.graph.name
        assert st["graphs"] == len(items)
        assert st["groups"] == len({_width_class(it.s) for it in items})
        assert st["seed_edge_traversals"] == plain_work
    for it in items[:6]:  # the oracle directly, on a few graphs
        want = oracle.run(it.graph, it.seeds)
        with pg.Batch() as b1:
            b1.add_inputs(it.graph, it.seeds)
            b1.run()
            got = b1.result(0)
        assert got.rounds == want["rounds"]
        assert np.array_equal(got.counts, want["counts"])
        assert np.array_equal(got.m_active, want["m_active"])
    # each graph's own m_active inside a packed batch, against the oracle
    with pg.Batch() as b:
        for it in items[:8]:
            b.add_inputs(it.graph, it.seeds)
        b.run()
        for k, it in enumerate(items[:8]):
            assert np.array_equal(b.result(k).m_active, oracle.run(it.graph, it.seeds)["m_active"])


def test_batch_result_independent_of_company():
    """A graph's counts are the same alone, in a batch, and in a batch in a
    different order (no bit crosses between packed graphs)."""
    items = _mix()[:10]
    runs = []
    for order in (list(range(10)), list(range(9, -1, -1))):
        with pg.Batch() as b:
            pos = {k: b.add_inputs(items[k].graph, items[k].seeds) for k in order}
            b.run()
            runs.append({k: b.result(pos[k]) for k in order})
    for k in range(10):
        assert runs[0][k].rounds == runs[1][k].rounds
        assert np.array_equal(runs[0][k].counts, runs[1][k].counts)
        assert np.array_equal(runs[0][k].m_active, runs[1][k].m_active)


def test_batch_edge_cases():
    """Isolated nodes, a single-node graph, a long path (many more rounds
    than its company), s = n, and a rerun after adding a graph."""
    p = I.path(300, directed=True)
    lone = I.from_arcs(1, [], [])
    iso = I.from_arcs(50, [0, 1], [1, 2])
    k5 = I.complete(5)
    cases = [(p, np.array([0, 150, 299], np.int32)), (lone, np.array([0], np.int32)),
             (iso, I.seeds(50, 50, 9)), (k5, np.arange(5, dtype=np.int32))]
    with pg.Batch() as b:
        for g, sd in cases:
            b.add_inputs(g, sd)
        b.run()
        for k, (g, sd) in enumerate(cases):
            want = oracle.run(g, sd)
            got = b.result(k)
            assert got.rounds == want["rounds"], g.name
            assert np.array_equal(got.counts, want["counts"]), g.name
            assert np.array_equal(got.m_active, want["m_active"]), g.name
        g2 = I.cycle(40)
        k2 = b.add_inputs(g2, np.array([3, 17], np.int32))
        b.run()
        want = oracle.run(g2, np.array([3, 17], np.int32))
        assert np.array_equal(b.result(k2).counts, want["counts"])
        assert np.array_equal(b.result(0).counts, oracle.run(p, cases[0][1])["counts"])


def test_batch_wide_signatures():
    """A width class above 8 words (s = 600 -> 10 words, padded to 16)."""
    g = I.er(3000, 6, 11)
    sd = I.seeds(g.n, 600, 12)
    g2 = I.grid(40, 40, 0.05, 13)
    sd2 = I.seeds(g2.n, 520, 14)
    with pg.Batch() as b:
        b.add_inputs(g, sd)
        b.add_inputs(g2, sd2)
        b.run()
        assert b.stats()["groups"] == 1
        for k, (gg, ss) in enumerate(((g, sd), (g2, sd2))):
            want = oracle.run(gg, ss)
            assert np.array_equal(b.result(k).counts, want["counts"])
            assert np.array_equal(b.result(k).m_active, want["m_active"])


def test_batch_rejects_bad_input():
    with pg.Batch() as b:
        g = I.er(100, 4, 1)
        with pytest.raises(pg.PropagateError):
            b.add_inputs(g, np.array([1, 1], np.int32))  # duplicate seed
        with pytest.raises(pg.PropagateError):
            b.add_inputs(g, np.array([100], np.int32))  # out of range
        with pytest.raises(pg.PropagateError):
            b.run()  # empty batch
        k = b.add_inputs(g, np.array([0, 5], np.int32))
        with pytest.raises(pg.PropagateError):
            b.result(k)  # no run yet


@pytest.mark.parametrize("direction", [pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
def test_batch_forced_direction(direction):
    """Every round dense (sliced-ELL chunks of finished graphs skipped) or
    every round sparse; a long path among short graphs of the same width."""
    items = list(_mix()[:12])
    extra = [(I.path(400, directed=True), np.array([0, 7, 399], np.int32)),
             (I.grid(60, 60, 0.05, 71), I.seeds(3600, 64, 72))]
    with pg.Batch() as b:
        for it in items:
            b.add_inputs(it.graph, it.seeds)
        for g, sd in extra:
            b.add_inputs(g, sd)
        b.run(opts=pg.options(direction=direction))
        for k, it in enumerate(items):
            want, _ = _plain(it)
            got = b.result(k)
            assert got.rounds == want.rounds and np.array_equal(got.counts, want.counts)
            assert np.array_equal(got.m_active, want.m_active)
        for j, (g, sd) in enumerate(extra):
            want = oracle.run(g, sd)
            got = b.result(len(items) + j)
            assert got.rounds == want["rounds"] and np.array_equal(got.counts, want["counts"])
            assert np.array_equal(got.m_active, want["m_active"])


@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_SPARSE])
def test_batch_push_rounds(direction):
    """sparse_push = 2 in a packed batch: in each round the graphs below
    their own dense threshold push (k_push, after the pull) while the others
    are swept whole; counts and rounds equal the plain runs', the work is the
    plain runs' work, and graphs of 8-word rows (s = 400, 512) push too."""
    items = list(_mix()[:12])
    extra = [(I.path(400, directed=True), np.array([0, 7, 399], np.int32)),
             (I.grid(60, 60, 0.05, 73), I.seeds(3600, 512, 74)),
             (I.rmat(11, 8, 75, directed=False), I.seeds(2048, 400, 76)),
             (I.er(2500, 5, 77), I.seeds(2500, 500, 78))]
    with pg.Batch() as b:
        for it in items:
            b.add_inputs(it.graph, it.seeds)
        for g, sd in extra:
            b.add_inputs(g, sd)
        b.run(opts=pg.options(direction=direction, sparse_push=2))
        work = b.stats()["seed_edge_traversals"]
        plain_work = 0
        for k, it in enumerate(items):
            want, w = _plain(it)
            plain_work += w
            got = b.result(k)
            assert got.rounds == want.rounds and np.array_equal(got.counts, want.counts)
            assert np.array_equal(got.m_active, want.m_active)
        for j, (g, sd) in enumerate(extra):
            want = oracle.run(g, sd)
            G = pg.Graph.from_inputs(g)
            pg.propagate_p(G, sd)
            plain_work += G.last_stats()["seed_edge_traversals"]
            G.close()
            got = b.result(len(items) + j)
            assert got.rounds == want["rounds"] and np.array_equal(got.counts, want["counts"])
            assert np.array_equal(got.m_active, want["m_active"])
        assert work == plain_work


def test_batch_large_graph_runs_alone():
    """A graph whose four signature arrays fill half of L2 (a 600^2 grid with
    s = 300: 360,000 nodes x 8 words) runs alone, as a group of its own
    through the single-graph path, beside the packed small graphs of the
    batch: its counts equal the oracle's, every small graph's the plain
    run's, and the batch's work is the plain runs' work."""
    big = I.grid(600, 600, 0.05, 81)
    sb = I.seeds(big.n, 300, 82)
    items = list(_mix()[:8])
    with pg.Batch() as b:
        for it in items:
            b.add_inputs(it.graph, it.seeds)
        kb = b.add_inputs(big, sb)
        b.run()
        st = b.stats()
        assert st["groups"] == len({_width_class(it.s) for it in items}) + 1
        alone = [ng for ng, _ in b.group_options()]
        assert alone.count(1) >= 1
        hist, _ = oracle.seed_histograms(big, sb, cap=6000)
        got = b.result(kb)
        assert got.rounds == hist.shape[1] - 1
        assert np.array_equal(got.counts, hist.T.astype(np.uint32))
        work = 0
        for k, it in enumerate(items):
            want, w = _plain(it)
            work += w
            assert np.array_equal(b.result(k).counts, want.counts)
        G = pg.Graph.from_inputs(big)
        alone_res = pg.propagate_p(G, sb)
        work += G.last_stats()["seed_edge_traversals"]
        G.close()
        assert st["seed_edge_traversals"] == work
        assert np.array_equal(got.m_active, alone_res.m_active)  # the solo group's own


def test_batch_streams_give_the_same_counts():
    """Groups run one after another, four at a time and sixteen at a time:
    the same counts and work (each group's propagation is independent)."""
    items = list(_mix()[:20])
    extra = (I.grid(520, 520, 0.05, 91), I.seeds(270_400, 500, 92))  # runs alone
    runs = []
    with pg.Batch() as b:
        for it in items:
            b.add_inputs(it.graph, it.seeds)
        b.add_inputs(*extra)
        for k in (1, 4, 16):
            b.set_streams(k)
            b.run()
            runs.append(([b.result(i).counts for i in range(len(items) + 1)],
                         b.stats()["seed_edge_traversals"],
                         [b.result(i).m_active for i in range(len(items) + 1)]))
    for counts, work, mact in runs[1:]:
        assert work == runs[0][1]
        for a, c in zip(runs[0][0], counts):
            assert np.array_equal(a, c)
        for a, c in zip(runs[0][2], mact):
            assert np.array_equal(a, c)
    want, _ = _plain(items[0])
    assert np.array_equal(runs[0][0][0], want.counts)


@pytest.mark.parametrize("window_rows", [5, 64])
def test_batch_m_active_across_window_shifts(window_rows):
    """Each graph's m_active in a packed batch whose counts window holds only
    a few rounds at a time (the per-graph slots move with it, the next
    round's claims carried over), in pull and push rounds, against the oracle:
    a 400-node path (400 rounds) beside short graphs, a grid, an R-MAT with
    hub rows cut into pieces, and graphs whose last rounds differ."""
    cases = [(I.path(400, directed=True), np.array([0, 7, 399], np.int32)),
             (I.grid(50, 40, 0.05, 101), I.seeds(2000, 64, 102)),
             (I.rmat(12, 8, 103, directed=True), I.seeds(4096, 64, 104)),
             (I.er(3000, 4, 105), I.seeds(3000, 50, 106)),
             (I.cycle(90), np.array([3, 40], np.int32))]
    wants = [oracle.run(g, sd) for g, sd in cases]
    for push in (1, 2):
        with pg.Batch() as b:
            for g, sd in cases:
                b.add_inputs(g, sd)
            b.run(opts=pg.options(window_rows=window_rows, sparse_push=push))
            assert b.stats()["groups"] == 1
            for k, ((g, _), want) in enumerate(zip(cases, wants)):
                got = b.result(k)
                assert got.rounds == want["rounds"], g.name
                assert np.array_equal(got.counts, want["counts"]), g.name
                assert np.array_equal(got.m_active, want["m_active"]), (g.name, push)
