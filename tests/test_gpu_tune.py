"""Autotuner (pg_autotune, pg_batch_tune) and the schedule knobs it turns:
every words-per-thread / lanes / threshold / changed-test choice gives
bit-identical counts (checked against the oracle), and the tuner returns
options whose counts equal the defaults'."""
import functools

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _case(s):
    g = I.rmat(13, 12, 41, directed=True)
    seeds = I.seeds(g.n, s, 42)
    return g, seeds, oracle.run(g, seeds)


@pytest.mark.parametrize("s,wpt", [(256, 1), (256, 2), (256, 4), (512, 2), (512, 4),
                                   (512, 8), (700, 4), (128, 1)])
@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
def test_words_per_thread_schedules_identical(s, wpt, direction):
    g, seeds, want = _case(s)
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, seeds, opts=pg.options(words_per_thread=wpt, direction=direction))
    assert res.rounds == want["rounds"]
    assert np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, want["m_active"])


def test_words_per_thread_rejects_bad_values():
    g, seeds, _ = _case(256)
    G = pg.Graph.from_inputs(g)
    for bad in (3, 16, -1):
        with pytest.raises(pg.PropagateError):
            pg.propagate_p(G, seeds, opts=pg.options(words_per_thread=bad))


def test_autotune_keeps_counts():
    g, seeds, want = _case(256)
    G = pg.Graph.from_inputs(g)
    o, rep = pg.autotune(G, seeds, max_trials=12)
    assert 1 <= rep["trials"] <= 12
    assert rep["best_ms"] <= rep["default_ms"] + 1e-9
    res = pg.propagate_p(G, seeds, opts=o)
    assert np.array_equal(res.counts, want["counts"])
    d = pg.options_dict(o)
    assert d["words_per_thread"] in (0, 1, 2, 4)
    assert d["group_lanes"] in (0, 1, 2, 4, 8, 16, 32)


def test_autotune_propagate_s_keeps_counts():
    g, seeds, want = _case(256)
    G = pg.Graph.from_inputs(g)
    o, rep = pg.autotune(G, seeds, max_trials=10, algorithm="s")
    assert 1 <= rep["trials"] <= 10
    res = pg.propagate_s(G, seeds, opts=o)
    assert np.array_equal(res.counts, want["counts"])
    assert pg.options_dict(o)["passes_together"] in (0, 1, 2, 4)


def test_batch_tune_then_run():
    items = I.mix(16, 500, 20_000, 8)
    with pg.Batch() as b:
        for it in items:
            b.add_inputs(it.graph, it.seeds)
        rep = b.tune(max_trials=6)
        assert rep["trials"] >= 1
        b.run()  # tuned options
        groups = b.group_options()
        assert sum(ng for ng, _ in groups) == len(items)
        for k, it in enumerate(items):
            want = oracle.run(it.graph, it.seeds)
            got = b.result(k)
            assert got.rounds == want["rounds"]
            assert np.array_equal(got.counts, want["counts"])


# ------------------------------------------------------------ wide rows
@functools.lru_cache(maxsize=None)
def _wide_case(kind, s):
    if kind == "rmat":  # hubs: rows longer than one 256-arc piece
        g = I.rmat(14, 16, 51, directed=True)
    else:
        g = I.er(12_000, 10, 52)
    seeds = I.seeds(g.n, s, 53)
    return g, seeds, oracle.run(g, seeds)


@pytest.mark.parametrize("kind,s", [("rmat", 520), ("rmat", 1024), ("er", 2047), ("rmat", 2100),
                                    ("er", 4100), ("rmat", 6000), ("er", 8200)])
@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
def test_wide_rows_identical(kind, s, direction):
    """Every words-per-lane class of the wide kernel (1-4 words in registers,
    and the generic passes above 128 words), split rows, both round kinds."""
    g, seeds, want = _wide_case(kind, s)
    G = pg.Graph.from_inputs(g)
    for wide in (0, 2):
        res = pg.propagate_p(G, seeds, opts=pg.options(direction=direction, wide_rows=wide))
        assert res.rounds == want["rounds"], wide
        assert np.array_equal(res.counts, want["counts"]), wide
        assert np.array_equal(res.m_active, want["m_active"]), wide


def test_wide_rows_in_batch_and_server():
    g, seeds, want = _wide_case("er", 2047)
    g2, seeds2, want2 = _wide_case("rmat", 2100)
    with pg.Batch() as b:
        b.add_inputs(g, seeds)
        b.add_inputs(g2, seeds2)
        b.run()
        assert np.array_equal(b.result(0).counts, want["counts"])
        assert np.array_equal(b.result(1).counts, want2["counts"])
    with pg.Server(slots=2) as srv:
        a = srv.submit(srv.add_inputs(g), seeds)
        c = srv.submit(srv.add_inputs(g2), seeds2)
        assert np.array_equal(srv.result(a)[0].counts, want["counts"])
        assert np.array_equal(srv.result(c)[0].counts, want2["counts"])


# ------------------------------------------------ PROPAGATE-S passes together
def _oracle_s_mactive(g, seeds, planes, rounds):
    _, _, dmat = oracle.seed_histograms(g, seeds, with_distances=True)
    total = np.zeros(rounds + 2, dtype=np.uint64)
    for b in range(0, len(seeds), planes):
        sub = np.ascontiguousarray(dmat[:, b:b + planes])
        part = oracle.m_active(g, sub, int(sub.max()) + 1)
        total[:part.size] += part
    return total


@pytest.mark.parametrize("planes", [64, 17, 1])
@pytest.mark.parametrize("together", [1, 2, 3, 0])
def test_s_passes_together_identical(planes, together):
    g = I.rmat(12, 10, 81, directed=True)
    seeds = I.seeds(g.n, 150, 82)
    want = oracle.run(g, seeds)
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_s(G, seeds, opts=pg.options(planes_per_pass=planes,
                                                   passes_together=together))
    assert res.rounds == want["rounds"]
    assert np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, _oracle_s_mactive(g, seeds, planes, want["rounds"]))
    st = G.last_stats()
    assert st["passes"] == -(-150 // planes)


# ------------------------------------------------------ progressive sampling
def test_progressive_sampling():
    """Blocks of seeds until the Thm. 3 sample size: the counts equal the
    oracle's for the drawn seeds, and the estimates approach the exact
    all-pairs values (s = n) within eps."""
    g = I.er(3000, 8, 101)
    eps = 0.1
    G = pg.Graph.from_inputs(g)
    res, seeds, hist = pg.progressive(G, eps, rng_seed=5, block=200)
    assert res.s == len(seeds) == min(g.n, int(np.ceil(np.log(g.n) / eps ** 2)))
    assert len(set(seeds.tolist())) == len(seeds)
    want = oracle.run(g, seeds)
    assert np.array_equal(res.counts, want["counts"])
    exact = oracle.run(g, np.arange(g.n, dtype=np.int32))["metrics"]
    est = pg.metrics(res, g.n)
    assert abs(est["avg_distance"] - exact["avg_distance"]) <= eps * exact["avg_distance"]
    assert hist[-1]["seeds"] == res.s and len(hist) == -(-res.s // 200)
    # stability rule: stops earlier, still a prefix of the same draw
    res2, seeds2, hist2 = pg.progressive(G, eps, rng_seed=5, block=200, stable_tol=0.05)
    assert res2.s <= res.s and np.array_equal(seeds2, seeds[:res2.s])
    assert np.array_equal(res2.counts[:, :], oracle.run(g, seeds2)["counts"])


def test_exact_mode_wide_rows():
    """s = n on 3,000 nodes (47 words per node): PROPAGATE-P through the wide
    kernel, PROPAGATE-S as 47 passes run together over replicas; metrics
    from all pairs."""
    g = I.er(3000, 6, 111)
    seeds = np.arange(g.n, dtype=np.int32)
    want = oracle.run(g, seeds)
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_p(G, seeds)
    assert G.last_stats()["words_per_gather"] == 0  # the wide-row kernel
    assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, want["m_active"])
    res_s = pg.propagate_s(G, seeds)
    assert np.array_equal(res_s.counts, want["counts"])
    m = pg.metrics(res, g.n)
    assert m["R_last"] == want["metrics"]["R_last"]


def test_exact_mode_313_words():
    """s = n on 20,000 nodes: 313 words per node, so the wide-row kernel
    sweeps each row in several 32-words-per-lane passes; P, S and the
    all-pairs metrics match the oracle."""
    g = I.er(20_000, 8, 121)
    seeds = np.arange(g.n, dtype=np.int32)
    want = oracle.run(g, seeds)
    G = pg.Graph.from_inputs(g)
    for direction in (pg.PG_DIR_AUTO, pg.PG_DIR_SPARSE):
        res = pg.propagate_p(G, seeds, opts=pg.options(direction=direction))
        assert G.last_stats()["words_per_gather"] == 0
        assert res.rounds == want["rounds"] and np.array_equal(res.counts, want["counts"])
        assert np.array_equal(res.m_active, want["m_active"])
    res_s = pg.propagate_s(G, seeds)
    assert np.array_equal(res_s.counts, want["counts"])
    m = pg.metrics(res, g.n)
    for k in ("R_last", "avg_distance"):
        assert m[k] == pytest.approx(want["metrics"][k], rel=1e-12)


# ------------------------------------------- PROPAGATE-S passes as words
@functools.lru_cache(maxsize=None)
def _pw_case(kind):
    if kind == "rmat":  # hubs: rows cut into pieces
        g = I.rmat(12, 10, 91, directed=True)
    elif kind == "grid":  # many rounds: passes end at different rounds
        g = I.grid(40, 40, 0.05, 92)
    else:
        g = I.er(3000, 6, 93)
    seeds = I.seeds(g.n, 300, 94)  # 5 passes, the last of 44 seeds
    want = oracle.run(g, seeds)
    return g, seeds, want, _oracle_s_mactive(g, seeds, 64, want["rounds"])


@pytest.mark.parametrize("kind", ["rmat", "grid", "er"])
@pytest.mark.parametrize("words", [2, 4, 8])
@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
def test_s_pass_words_identical(kind, words, direction):
    """Passes side by side as signature words: counts and rounds as the
    oracle's, m_active as the passes' own, summed (skip rule per pass), with
    sparse rounds pushed (k_push, claims per pass; rows gathered whole) and
    pulled (the post kernel's claims)."""
    g, seeds, want, mact = _pw_case(kind)
    G = pg.Graph.from_inputs(g)
    # lanes 1: many rows in pieces; words_per_thread below the row: pulled
    for lanes, wpt, push in ((0, 0, 0), (0, 0, 1), (1, 0, 0), (1, 0, 1), (1, 1, 0), (4, 2, 0)):
        res = pg.propagate_s(G, seeds, opts=pg.options(pass_words=words, direction=direction,
                                                       group_lanes=lanes, words_per_thread=wpt,
                                                       sparse_push=push))
        case = (lanes, wpt, push)
        assert res.rounds == want["rounds"], case
        assert np.array_equal(res.counts, want["counts"]), case
        assert np.array_equal(res.m_active, mact), case
        assert G.last_stats()["passes"] == 5


def test_s_pass_words_rejects_bad_values():
    g, seeds, _, _ = _pw_case("er")
    G = pg.Graph.from_inputs(g)
    for bad in (-1, -64):
        with pytest.raises(pg.PropagateError):
            pg.propagate_s(G, seeds, opts=pg.options(pass_words=bad))


@functools.lru_cache(maxsize=None)
def _wide_mact(kind, s):
    g, seeds, want = _wide_case(kind, s)
    return _oracle_s_mactive(g, seeds, 64, want["rounds"])


@pytest.mark.parametrize("kind,s", [("rmat", 600), ("rmat", 2100), ("er", 8200)])
@pytest.mark.parametrize("direction", [pg.PG_DIR_AUTO, pg.PG_DIR_DENSE, pg.PG_DIR_SPARSE])
def test_s_pass_words_wide(kind, s, direction):
    """All passes at once as the words of one wide signature (the wide-row
    kernel: registers for 10 and 33 words, 128-word sweeps for 129), rows
    cut into pieces on the R-MAT hubs: counts and per-pass m_active."""
    g, seeds, want = _wide_case(kind, s)
    G = pg.Graph.from_inputs(g)
    res = pg.propagate_s(G, seeds, opts=pg.options(direction=direction))
    st = G.last_stats()
    assert st["pass_words"] == -(-s // 64) and st["words_per_gather"] == 0
    assert res.rounds == want["rounds"]
    assert np.array_equal(res.counts, want["counts"])
    assert np.array_equal(res.m_active, _wide_mact(kind, s))
    # a few passes at a time: the same
    res2 = pg.propagate_s(G, seeds, opts=pg.options(direction=direction, pass_words=3))
    assert np.array_equal(res2.counts, want["counts"])
    assert np.array_equal(res2.m_active, _wide_mact(kind, s))


def test_wide_rows_across_counts_windows():
    """A counts window of 3 rounds on a grid of ~120 rounds, rows of 33 and
    16 words: the window shifts many times, and the wide post kernel's
    per-row bit counts (which decide saturation, hence m_active) carry
    across the shifts."""
    g = I.grid(60, 60, 0.05, 131)
    for s in (2100, 1000):
        seeds = I.seeds(g.n, s, 132)
        want = oracle.run(g, seeds)
        assert want["rounds"] > 30
        G = pg.Graph.from_inputs(g)
        for use_graphs in (1, 0):
            res = pg.propagate_p(G, seeds, opts=pg.options(window_rows=3, use_graphs=use_graphs))
            assert res.rounds == want["rounds"]
            assert np.array_equal(res.counts, want["counts"])
            assert np.array_equal(res.m_active, want["m_active"])
