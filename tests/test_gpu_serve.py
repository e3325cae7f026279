"""Serving loop (pg_server_*): each request's counts are the same alone
(pg_propagate_p on its own graph handle) and in the mix, whatever it was
merged with, whichever slot ran it and whenever it arrived; admission keeps
the charged device memory within the budget; queued requests on one graph
are merged, and requests on graphs of one signature width run as a packed
union; cancel and remove behave as documented."""
import functools
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import _abi
from paper_2301_06499_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _pool():
    return [it.graph for it in I.mix(8, 500, 30_000, 5)]


def _alone(g, seeds):
    G = pg.Graph.from_inputs(g)
    try:
        return pg.propagate_p(G, seeds)
    finally:
        G.close()


def _requests(count, seed):
    """(pool index, seeds) pairs: s from 1 to 700, seeds drawn per request,
    so that requests on one graph overlap in their seed nodes."""
    pool = _pool()
    out = []
    for k in range(count):
        gi = int(I.rand(seed, 1, k) % len(pool))
        n = pool[gi].n
        s = int(min(n, (1, 37, 64, 128, 200, 256, 512, 700)[I.rand(seed, 2, k) % 8]))
        out.append((gi, I.seeds(n, s, seed * 7919 + k)))
    return out


def _check_same(g, seeds, res):
    want = _alone(g, seeds)
    assert res.rounds == want.rounds
    assert np.array_equal(res.counts, want.counts)


def test_burst_same_alone_and_in_mix():
    pool = _pool()
    reqs = _requests(60, 11)
    with pg.Server(slots=4) as srv:
        gids = [srv.add_inputs(g) for g in pool]
        rids = [srv.submit(gids[gi], sd) for gi, sd in reqs]
        infos = []
        for rid, (gi, sd) in zip(rids, reqs):
            res, info = srv.result(rid)
            infos.append(info)
            assert info["state"] == _abi.PG_REQ_DONE
            _check_same(pool[gi], sd, res)
        st = srv.stats()
    assert st["completed"] == 60 and st["failed"] == 0
    assert st["propagations"] <= 60
    assert st["gpu_launches"] >= 3 * st["propagations"]  # set-up kernels + rounds
    assert max(i["merged"] for i in infos) >= 1
    assert st["peak_bytes"] <= st["budget_bytes"]


def test_queued_requests_on_one_graph_are_merged():
    """One slot busy with a long propagation; five requests on another graph
    queue behind it (two of them sharing seed nodes) and run as one."""
    long_g = I.grid(800, 800, 0.05, 21)
    g = _pool()[0]
    sets = [I.seeds(g.n, s, 100 + k) for k, s in enumerate((64, 100, 3, 256, 64))]
    sets[4] = sets[0].copy()  # identical seed set
    with pg.Server(slots=1, cross_graph=False) as srv:
        lg = srv.add_inputs(long_g)
        gid = srv.add_inputs(g)
        first = srv.submit(lg, I.seeds(long_g.n, 64, 5))
        rids = [srv.submit(gid, sd) for sd in sets]
        _, info0 = srv.result(first)
        for rid, sd in zip(rids, sets):
            res, info = srv.result(rid)
            assert info["merged"] == len(sets)
            _check_same(g, sd, res)
        assert srv.stats()["propagations"] == 2


def test_admission_within_budget():
    pool = _pool()
    reqs = _requests(30, 12)
    with pg.Server(slots=4) as probe:
        for g in pool:
            probe.add_inputs(g)
        resident = probe.stats()["resident_bytes"]
    # room for the graphs and little more than the largest request
    budget = resident + 64 * 1024 * 1024
    with pg.Server(slots=4, hbm_budget=budget) as srv:
        gids = [srv.add_inputs(g) for g in pool]
        rids = [srv.submit(gids[gi], sd) for gi, sd in reqs]
        for rid, (gi, sd) in zip(rids, reqs):
            res, _ = srv.result(rid)
            _check_same(pool[gi], sd, res)
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        assert st["completed"] == 30
        # a request that cannot fit even alone is refused at submission
        big = I.er(200_000, 8, 3)
        with pytest.raises(pg.PropagateError) as e:
            srv.submit(srv.add_inputs(big), I.seeds(big.n, 4096, 1))
        assert e.value.status in (_abi.PG_ENOMEM,)


def test_cancel_and_remove():
    long_g = I.grid(800, 800, 0.05, 22)
    g = _pool()[1]
    with pg.Server(slots=1) as srv:
        lg = srv.add_inputs(long_g)
        gid = srv.add_inputs(g)
        first = srv.submit(lg, I.seeds(long_g.n, 64, 6))
        victim = srv.submit(gid, I.seeds(g.n, 64, 7))
        keep = srv.submit(gid, I.seeds(g.n, 32, 8))
        srv.cancel(victim)
        assert srv.poll(victim)["state"] == _abi.PG_REQ_CANCELLED
        with pytest.raises(pg.PropagateError) as e:
            srv.result(victim)
        assert e.value.status == _abi.PG_ECANCELLED
        with pytest.raises(pg.PropagateError):
            srv.remove_graph(gid)  # a request is still queued on it
        srv.result(first)
        res, info = srv.result(keep)
        assert info["merged"] == 1
        _check_same(g, I.seeds(g.n, 32, 8), res)
        srv.remove_graph(gid)
        with pytest.raises(pg.PropagateError):
            srv.submit(gid, I.seeds(g.n, 4, 1))
        st = srv.stats()
        assert st["cancelled"] == 1 and st["graphs"] == 1


def test_poisson_arrivals_from_another_thread():
    """Requests arrive at ~1000/s from a producer thread while the main
    thread collects results: every answer equals the request alone, and the
    latencies are consistent (submit <= start <= done)."""
    pool = _pool()
    reqs = _requests(150, 13)
    rng = np.random.default_rng(0)
    gaps = rng.exponential(1.0 / 1000.0, size=len(reqs))
    with pg.Server(slots=4) as srv:
        gids = [srv.add_inputs(g) for g in pool]
        rids = [None] * len(reqs)
        ready = threading.Semaphore(0)

        def produce():
            for k, (gi, sd) in enumerate(reqs):
                time.sleep(gaps[k])
                rids[k] = srv.submit(gids[gi], sd)
                ready.release()

        th = threading.Thread(target=produce)
        th.start()
        lat = []
        for k, (gi, sd) in enumerate(reqs):
            ready.acquire()
            res, info = srv.result(rids[k])
            assert info["submit_ns"] <= info["start_ns"] <= info["done_ns"]
            lat.append((info["done_ns"] - info["submit_ns"]) / 1e6)
            _check_same(pool[gi], sd, res)
        th.join()
    assert np.percentile(lat, 99) >= np.percentile(lat, 50) > 0


def test_server_matches_oracle():
    g = I.rmat(12, 8, 31, directed=True)
    sd = I.seeds(g.n, 130, 32)
    want = oracle.run(g, sd)
    with pg.Server(slots=2) as srv:
        gid = srv.add_inputs(g)
        a = srv.submit(gid, sd)
        b = srv.submit(gid, sd[:7])
        res, _ = srv.result(a)
        res_b, _ = srv.result(b)
    assert res.rounds == want["rounds"]
    assert np.array_equal(res.counts, want["counts"])
    wb = oracle.run(g, sd[:7])
    assert np.array_equal(res_b.counts, wb["counts"])


def test_server_rejects_bad_requests():
    g = _pool()[2]
    with pg.Server(slots=1) as srv:
        gid = srv.add_inputs(g)
        for bad in (np.array([0, 0], np.int32), np.array([g.n], np.int32),
                    np.array([-1], np.int32)):
            with pytest.raises(pg.PropagateError):
                srv.submit(gid, bad)
        with pytest.raises(pg.PropagateError):
            srv.submit(gid + 17, np.array([0], np.int32))
        rid = srv.submit(gid, np.array([1, 2], np.int32))
        assert srv.wait(rid, 10_000)["state"] == _abi.PG_REQ_DONE


def test_requests_on_different_graphs_run_as_one_union():
    """One slot busy with a long propagation; requests queue behind it on
    five graphs (a relabelled R-MAT, a digraph, a grid, an ER graph and a
    small mixed one). Those of one signature width (two words) are merged
    across graphs into a packed union; a wider request runs on its own.
    Every answer equals the request alone."""
    long_g = I.grid(800, 800, 0.05, 31)
    graphs = [I.rmat(17, 8, 32, directed=False), I.rmat(12, 16, 33, directed=True),
              I.grid(120, 90, 0.05, 34), I.er(5000, 6, 35), _pool()[1]]
    reqs = []
    for k, g in enumerate(graphs):
        for j, sz in enumerate((100, 70)):  # two words each
            reqs.append((k, I.seeds(g.n, sz, 40 + 10 * k + j)))
    reqs.append((0, I.seeds(graphs[0].n, 300, 99)))  # five words: another width
    with pg.Server(slots=1) as srv:
        lg = srv.add_inputs(long_g)
        gids = [srv.add_inputs(g) for g in graphs]
        first = srv.submit(lg, I.seeds(long_g.n, 512, 5))
        rids = [srv.submit(gids[k], sd) for k, sd in reqs]
        srv.result(first)
        merged = []
        for rid, (k, sd) in zip(rids, reqs):
            res, info = srv.result(rid)
            merged.append(info["merged"])
            _check_same(graphs[k], sd, res)
        st = srv.stats()
    assert max(merged[:-1]) > 2  # more requests in one run than any one graph had
    assert st["propagations"] < 1 + len(reqs)
    assert st["completed"] == 1 + len(reqs) and st["failed"] == 0
