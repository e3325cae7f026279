"""Pins for the CPU oracle, against things other than itself: Floyd-Warshall,
closed forms, a brute-force set simulation, hand-worked examples and the
paper's printed Twitch value. CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2301_06499_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = v
    return out


def _exact(g):
    """Oracle run in exact mode (every node a seed)."""
    seeds = np.arange(g.n, dtype=np.int32)
    hist, _ = oracle.seed_histograms(g, seeds)
    return hist, oracle.metrics(hist, g.n)


# ------------------------------------------------------------ BFS vs APSP
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("directed", [True, False])
def test_histograms_match_floyd_warshall(seed, directed):
    n = 5 + 9 * seed
    if directed:
        g = I.random_digraph(n, 2 * n, seed)
    else:
        g = I.er(n, 2.5, seed)
    dist = oracle.apsp_floyd_warshall(g)
    hist, ecc = oracle.seed_histograms(g, np.arange(n, dtype=np.int32))
    T = hist.shape[1] - 1
    for x in range(n):
        row = dist[x]
        want = np.bincount(row[row >= 0], minlength=T + 1)
        assert np.array_equal(hist[x], want[:T + 1])
        assert ecc[x] == row.max()


def test_histograms_sampled_subset_equals_rows_of_exact():
    g = I.random_digraph(40, 90, 11)
    full, _ = oracle.seed_histograms(g, np.arange(40, dtype=np.int32))
    pick = np.array([7, 3, 31, 0], dtype=np.int32)
    sub, _ = oracle.seed_histograms(g, pick)
    for i, x in enumerate(pick):
        assert np.array_equal(sub[i], full[x][:sub.shape[1]])


# --------------------------------------------------------- edge direction
def test_direction_forward_from_seed():
    # directed path 0 -> 1 -> 2 -> 3: the ball of seed 0 grows forward.
    g = I.path(4, directed=True)
    hist, ecc = oracle.seed_histograms(g, np.array([0, 3], dtype=np.int32))
    assert hist.shape == (2, 4)
    assert list(hist[0]) == [1, 1, 1, 1]
    assert list(hist[1]) == [1, 0, 0, 0]
    assert list(ecc) == [3, 0]


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [2, 3, 7, 10, 33])
def test_path_closed_form(n):
    _, m = _exact(I.path(n))
    assert m["diameter"] == n - 1
    assert m["avg_distance"] == pytest.approx((n + 1) / 3, rel=1e-13)
    assert m["connectivity_rate"] == pytest.approx(1.0, rel=1e-15)
    assert m["reachable_pairs"] == n * n


@pytest.mark.parametrize("n", [3, 4, 9, 10, 31, 32])
def test_cycle_closed_form(n):
    _, m = _exact(I.cycle(n))
    k = n // 2
    assert m["diameter"] == k
    want = (k + 1) / 2 if n % 2 else k * k / (2 * k - 1)
    assert m["avg_distance"] == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("n", [3, 5, 12])
def test_star_closed_form(n):
    _, m = _exact(I.star(n))
    assert m["diameter"] == 2
    assert m["avg_distance"] == pytest.approx(2 * (n - 1) / n, rel=1e-13)


@pytest.mark.parametrize("n", [2, 6, 17])
def test_complete_closed_form(n):
    _, m = _exact(I.complete(n))
    assert m["diameter"] == 1
    assert m["avg_distance"] == 1.0
    assert m["eff_diameter"] == 1


@pytest.mark.parametrize("a,b", [(2, 3), (4, 4), (3, 7), (5, 6)])
def test_grid_closed_form(a, b):
    g = I.grid(a, b, 0.0, 0)
    _, m = _exact(g)
    assert m["diameter"] == a + b - 2
    want = (b * (a * a - 1) + a * (b * b - 1)) / (3 * (a * b - 1))
    assert m["avg_distance"] == pytest.approx(want, rel=1e-13)
    assert m["connectivity_rate"] == pytest.approx(1.0, rel=1e-15)
    assert m["reachable_pairs"] == (a * b) ** 2


@pytest.mark.parametrize("n", [2, 5, 20])
def test_directed_path_connectivity_half(n):
    _, m = _exact(I.path(n, directed=True))
    assert m["connectivity_rate"] == pytest.approx(0.5, rel=1e-14)
    # ordered pairs u<v at distance v-u: mean (n+1)/3 as in the undirected case
    assert m["avg_distance"] == pytest.approx((n + 1) / 3, rel=1e-13)


@pytest.mark.parametrize("n", [2, 3, 8, 25])
def test_directed_star_closed_form(n):
    """Arcs from a centre to n-1 leaves (and the same arcs reversed), every
    node a seed: the centre's ball holds every leaf at distance 1 (out-star)
    or no other node (in-star), a leaf's ball the reverse. Either way
    R = [n, 2n-1]: diameter 1, mean distance 1, alpha = (n-1)/(n(n-1)) = 1/n,
    reachable pairs 2n-1, and the interpolated 90% effective diameter
    (0.9(2n-1) - n)/(n-1)."""
    leaves = np.arange(1, n, dtype=np.int32)
    centre = np.zeros(n - 1, dtype=np.int32)
    for src, dst, centre_row in ((centre, leaves, [1, n - 1]), (leaves, centre, [1, 0])):
        hist, m = _exact(I.from_arcs(n, src, dst))
        assert list(hist[0]) == centre_row
        assert all(list(hist[v]) == [1, 1 - centre_row[1] // (n - 1)] for v in range(1, n))
        assert m["diameter"] == 1 and m["eff_diameter"] == 1
        assert m["R_last"] == 2 * n - 1
        assert m["avg_distance"] == 1.0
        assert m["avg_distance_incl_self"] == pytest.approx((n - 1) / (2 * n - 1), rel=1e-15)
        assert m["connectivity_rate"] == pytest.approx(1.0 / n, rel=1e-15)
        assert m["reachable_pairs"] == 2 * n - 1
        assert m["eff_diameter_interp"] == pytest.approx((0.9 * (2 * n - 1) - n) / (n - 1),
                                                         rel=1e-13)


def test_isolated_nodes():
    g = I.from_arcs(5, np.array([], np.int32), np.array([], np.int32))
    hist, m = _exact(g)
    assert hist.shape == (5, 1)
    assert m["diameter"] == 0 and m["eff_diameter"] == 0
    assert m["connectivity_rate"] == 0.0 and m["avg_distance"] == 0.0
    assert m["reachable_pairs"] == 5.0


# -------------------------------------------------------- worked examples
def test_p4_worked_example():
    gold = _read_golden("p4_neighbourhood.txt")
    hist, m = _exact(I.path(4))
    R = np.cumsum(hist.sum(axis=0))
    assert list(R) == [int(x) for x in gold["R"]]
    assert m["eff_diameter"] == int(gold["eff_diameter"][0])
    assert m["eff_diameter_interp"] == pytest.approx(float(gold["eff_diameter_interp"][0]),
                                                     rel=1e-13)
    assert m["avg_distance"] == pytest.approx(float(gold["avg_distance"][0]), rel=1e-15)
    assert m["diameter"] == int(gold["diameter"][0])
    assert m["R_last"] == 16


def test_twitch_reachable_pairs_counts_self_pairs():
    gold = _read_golden("twitch_reachable_pairs.txt")
    n = int(gold["n"][0])
    exact = int(gold["exact_reachable_pairs"][0])
    # The printed exact value is n^2: pairs (u, u) are counted.
    assert n * n == exact
    # The oracle follows that convention: a connected graph in exact mode
    # reports n^2, and the (u, u) pairs are what separates n^2 from n(n-1).
    for g in (I.cycle(11), I.grid(3, 5, 0.0, 0), I.complete(6)):
        _, m = _exact(g)
        assert m["reachable_pairs"] == g.n * g.n
        assert m["R_last"] == g.n * g.n


def test_eff_diameter_rational_threshold():
    # Histogram with R = [10, 90, 100]: tau*R[T] = 90 exactly. The integer
    # rule must take k = 1 (R[1] = 90 >= 90), which a float 0.9 could miss.
    hist = np.array([[10, 80, 10]], dtype=np.int64)
    m = oracle.metrics(hist, 1000, 9, 10)
    assert m["eff_diameter"] == 1
    m = oracle.metrics(hist, 1000, 1, 1)
    assert m["eff_diameter"] == 2  # tau = 1 gives the diameter


def test_sampled_scaling():
    g = I.er(300, 3.0, 5)
    seeds = I.seeds(g.n, 17, 9)
    hist, _ = oracle.seed_histograms(g, seeds)
    m = oracle.metrics(hist, g.n)
    R_last = int(hist.sum())
    assert m["R_last"] == R_last
    assert m["reachable_pairs"] == pytest.approx(g.n / 17 * R_last, rel=1e-15)
    assert m["connectivity_rate"] == pytest.approx((R_last - 17) / (17 * (g.n - 1)), rel=1e-15)


# ------------------------------------- brute-force synchronous simulation
def _simulate(g, seeds):
    """Alg. 1 with Python sets on a tiny graph: sig[v] = seeds reached. Returns
    per-round per-seed new-node counts, and per round the arcs of nodes that
    are unsaturated and have an in-neighbour that changed the round before."""
    n, s = g.n, len(seeds)
    rp, col = g.row_ptr, g.col
    sig = [set() for _ in range(n)]
    for i, x in enumerate(seeds):
        sig[x].add(i)
    changed = set(int(x) for x in seeds)
    counts = [[1] * s]
    m_act = [0]
    while True:
        new = []
        arcs = 0
        for v in range(n):
            acc = set(sig[v])
            ins = col[rp[v]:rp[v + 1]]
            for u in ins:
                acc |= sig[u]
            new.append(acc)
            if len(sig[v]) < s and any(int(u) in changed for u in ins):
                arcs += len(ins)
        m_act.append(arcs)
        row = [0] * s
        changed = set()
        for v in range(n):
            for i in new[v] - sig[v]:
                row[i] += 1
            if new[v] != sig[v]:
                changed.add(v)
        sig = new
        if not changed:
            break
        counts.append(row)
    return np.array(counts, dtype=np.int64), np.array(m_act, dtype=np.uint64)


@pytest.mark.parametrize("case", range(8))
def test_oracle_equals_set_simulation(case):
    if case % 2:
        g = I.random_digraph(12 + 3 * case, 30 + 5 * case, case)
    else:
        g = I.er(15 + 4 * case, 2.0 + 0.3 * case, case)
    s = 1 + (case * 5) % g.n
    seeds = I.seeds(g.n, s, 100 + case)
    counts, m_act = _simulate(g, seeds)
    res = oracle.run(g, seeds)
    assert res["rounds"] == counts.shape[0] - 1
    assert np.array_equal(res["counts"].astype(np.int64), counts)
    assert np.array_equal(res["m_active"], m_act)


def test_m_active_counts_saturation_and_frontier():
    # Undirected path 0-1-2, seed {1}: round 1 updates 0 and 2 (1 in-arc
    # each); node 1 is saturated (s = 1) and is skipped. Round 2 (empty):
    # nodes 0 and 2 are saturated; node 1 is saturated. So [0, 2, 0].
    g = I.path(3)
    res = oracle.run(g, np.array([1], np.int32))
    assert list(res["m_active"]) == [0, 2, 0]
    # Two seeds {0, 2}: round 1: node 1 (unsaturated, in-arcs from 0 and 2
    # which changed at 0) -> 2 arcs; nodes 0, 2 have in-neighbour 1 which did
    # not change at round 0 -> inactive. Round 2: 0 and 2 have in-neighbour 1
    # (changed at 1) and a missing bit -> 1 + 1 arcs; node 1 saturated.
    # Round 3: everyone saturated -> 0.
    res = oracle.run(g, np.array([0, 2], np.int32))
    assert res["rounds"] == 2
    assert list(res["m_active"]) == [0, 2, 2, 0]


def test_metrics_avg_distance_excludes_self_pairs_includes_in_alt():
    hist, m = _exact(I.path(5))
    num = sum(d * hist[:, d].sum() for d in range(hist.shape[1]))
    assert m["dist_sum"] == num
    assert m["avg_distance"] == pytest.approx(num / (25 - 5), rel=1e-15)
    assert m["avg_distance_incl_self"] == pytest.approx(num / 25, rel=1e-15)
    assert math.isclose(m["avg_distance"], 2.0)


# ------------------------------------------------ Alg. 1 on the host
@pytest.mark.parametrize("kind,s", [("rmat", 1), ("rmat", 100), ("rmat", 200), ("grid", 64),
                                    ("er", 130), ("path", 7), ("iso", 40)])
def test_host_alg1_equals_bfs(kind, s):
    """Alg. 1 swept on s-bit signatures gains, in round t, exactly the seeds
    at distance t: its per-seed counts are the BFS histograms (two
    independent statements of Sec. 4's collision count)."""
    g = {"rmat": lambda: I.rmat(10, 8, 71, directed=True),
         "grid": lambda: I.grid(25, 25, 0.05, 72),
         "er": lambda: I.er(1500, 5, 73),
         "path": lambda: I.path(60, directed=True),
         "iso": lambda: I.from_arcs(100, [0, 1, 5], [1, 2, 6])}[kind]()
    seeds = I.seeds(g.n, min(s, g.n), 74)
    counts, T, mact = oracle.propagate_p(g, seeds, with_m_active=True)
    want = oracle.run(g, seeds)
    assert T == want["rounds"]
    assert np.array_equal(counts, want["counts"])
    # m_active as the sweeps find it (changed flags, saturation) equals the
    # one restated from BFS distances
    assert np.array_equal(mact, want["m_active"])


def test_host_alg1_path_closed_form_and_errors():
    # directed path 0 -> 1 -> ... -> 9 from seed 0: one new node per round
    g = I.path(10, directed=True)
    counts, T = oracle.propagate_p(g, np.array([0], np.int32))
    assert T == 9 and counts[:, 0].tolist() == [1] * 10
    with pytest.raises(OverflowError):  # a round beyond cap still gains bits
        oracle.propagate_p(g, np.array([0], np.int32), cap=4)
    with pytest.raises(ValueError):  # a repeated seed
        oracle.propagate_p(g, np.array([3, 3], np.int32))
