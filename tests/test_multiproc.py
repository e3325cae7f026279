"""Multi-process host logic on CPU (gloo, world size 2): seed sharding of
one problem and the final count gather, and the benchmark's max/sum
reductions over ranks. Each rank computes its seed slice with the oracle
(the GPU kernels are exercised elsewhere); the gathered counts must equal
the whole problem's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2301_06499_gb300.shard import seed_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, s, out_dir):
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2301_06499_gb300 import inputs as I
    from paper_2301_06499_gb300.shard import gather_counts
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = I.rmat(10, 8, 61, directed=True)
    seeds = I.seeds(g.n, s, 62)
    lo, hi = seed_shard(s, rank, world)
    res = oracle.run(g, seeds[lo:hi]) if hi > lo else {"counts": np.zeros((1, 0), np.uint32)}
    full = gather_counts(res["counts"], world)
    np.save(os.path.join(out_dir, f"counts{rank}.npy"), full)
    # the benchmark's reductions over ranks
    mx = bench.reduce_max(float(rank + 1), world)
    sm = bench.reduce_sum(float(rank + 1), world)
    np.save(os.path.join(out_dir, f"red{rank}.npy"), np.array([mx, sm]))
    dist.barrier()
    dist.destroy_process_group()


def test_seed_shard_partition():
    for s in (1, 63, 64, 65, 200, 256, 1000):
        for world in (1, 2, 3, 4, 8):
            parts = [seed_shard(s, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == s
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            for a, b in parts:  # whole words; only the end of the seeds is ragged
                assert (a % 64 == 0 or a == s) and (b % 64 == 0 or b == s)


@pytest.mark.parametrize("s", [200, 64])
def test_gloo_two_ranks_gather_equals_whole(tmp_path, s):
    import oracle
    from paper_2301_06499_gb300 import inputs as I
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, s, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    g = I.rmat(10, 8, 61, directed=True)
    seeds = I.seeds(g.n, s, 62)
    want = oracle.run(g, seeds)["counts"]
    for r in range(world):
        got = np.load(tmp_path / f"counts{r}.npy")
        assert got.shape == want.shape
        assert np.array_equal(got, want)
        mx, sm = np.load(tmp_path / f"red{r}.npy")
        assert mx == 2.0 and sm == 3.0



def _failing_worker(rank, world, port, out_dir):
    """Rank 1 fails between its propagation and the final gather (an
    exception on the host, no device work in flight); rank 0 must learn of
    it from the gather, as an error within the process group's timeout, not
    hang in it."""
    import datetime
    import time

    import torch.distributed as dist

    import oracle
    from paper_2301_06499_gb300 import inputs as I
    from paper_2301_06499_gb300.shard import gather_counts
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    g = I.rmat(9, 8, 63, directed=True)
    lo, hi = seed_shard(128, rank, world)
    res = oracle.run(g, I.seeds(g.n, 128, 64)[lo:hi])
    if rank == 1:
        raise RuntimeError("rank 1 fails before the gather")
    t0 = time.monotonic()
    try:
        gather_counts(res["counts"], world)
        outcome = "no error"
    except Exception as e:  # the backend's error type varies by version
        outcome = "error: " + type(e).__name__
    with open(os.path.join(out_dir, "rank0.txt"), "w") as f:
        f.write(f"{outcome}\n{time.monotonic() - t0:.3f}\n")


def test_gloo_peer_failure_surfaces_as_an_error(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        if p.is_alive():  # never expected: stop it and fail the test
            p.kill()
            p.join()
            pytest.fail("a rank hung after its peer failed")
    assert procs[1].exitcode != 0
    outcome, secs = (tmp_path / "rank0.txt").read_text().split("\n")[:2]
    assert outcome.startswith("error"), outcome
    assert float(secs) < 60.0
