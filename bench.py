"""Benchmark of the PROPAGATE hot path on GB300.

One step = PROPAGATE-P (Alg. 1) and PROPAGATE-S (Alg. 2) over the same seeds
on the benchmark workload, to fixpoint, through the C ABI, plus the Sec. 3
metrics from the counts. Work per step is the method-defined seed-edge
traversal count: each of the two runs solves the problem whose work is
sum_t s * m_active(t) (m_active from the PROPAGATE-P run).

Default workload: directed R-MAT, scale 22 (4,194,304 nodes), edge factor 16,
(a, b, c, d) = (.57, .19, .19, .05), RNG seed 2, duplicates removed, CSR over
in-edges; s = 256 seeds (4 words per node), uniform without replacement (RNG
seed 2). --workload selects the other shapes (see WORKLOADS).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank runs its own
independent replica of the workload (its own seed sample), so the per-GPU
work is fixed as N grows (weak scaling); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "seed-edge traversals/s (s*m_active/round) batched vs plain, bit-exact; p99 ms"
UNIT = "seed-edge traversals/s"
L2_BYTES = 129 * 1024 * 1024

WORKLOADS = {
    # name: (generator kwargs, s, description)
    "rmat22_directed_s256": (dict(kind="rmat", scale=22, ef=16, seed=2, directed=True), 256,
                             "directed R-MAT scale 22, edge factor 16, s=256 (P and S)"),
    "er1e4_s64": (dict(kind="er", n=10_000, d=8, seed=0), 64,
                  "undirected ER n=10,000 avg degree 8, s=64"),
    "grid4096_s128": (dict(kind="grid", rows=4096, cols=4096, p=0.05, seed=3), 128,
                      "4096x4096 grid, 5% edges deleted, s=128"),
    "rmat26_undirected_s512": (dict(kind="rmat", scale=26, ef=16, seed=2, directed=False), 512,
                               "undirected R-MAT scale 26, edge factor 16, s=512"),
}
SEED_RNG = {"rmat22_directed_s256": 2, "er1e4_s64": 1, "grid4096_s128": 3,
            "rmat26_undirected_s512": 2}


def make_graph(spec):
    from paper_2301_06499_gb300 import inputs as I
    k = spec["kind"]
    if k == "rmat":
        return I.rmat(spec["scale"], spec["ef"], spec["seed"], directed=spec["directed"])
    if k == "er":
        return I.er(spec["n"], spec["d"], spec["seed"])
    return I.grid(spec["rows"], spec["cols"], spec["p"], spec["seed"])


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def seed_stream(workload: str, rank: int) -> int:
    """RNG seed of rank r's seed sample: rank 0 uses the workload's own."""
    return SEED_RNG[workload] + 1000 * rank


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl)
                          if f.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def pull_bytes(st: dict) -> float:
    """Algorithmic bytes of the pull kernel summed over a call's launches:
    per work item 8 B (list entry) + 16 B (row_ptr pair) + 8 Wp B (own
    signature); per arc scanned 4 B (column index); per neighbour signature
    ORed 8 Wp B; per changed row 8 Wp B (signature write)."""
    w = 8.0 * st["words_per_row"]
    return (st["items"] * (24.0 + w) + st["arcs_scanned"] * 4.0 + st["rows_gathered"] * w
            + st["changed_rows"] * w)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2301_06499_gb300 as pg
    from paper_2301_06499_gb300 import inputs as I

    spec, s, desc = WORKLOADS[args.workload]
    g = make_graph(spec)
    seeds = I.seeds(g.n, s, seed_stream(args.workload, rank))
    stream = torch.cuda.current_stream()
    sptr = __import__("ctypes").c_void_p(stream.cuda_stream)
    G = pg.Graph.from_inputs(g, stream=sptr)
    opts_time = pg.options(timing=1)
    opts_run = pg.options(use_graphs=0 if args.plain_launches else 1)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def step(opts):
        rp = pg.propagate_p(G, seeds, opts=opts, stream=sptr)
        stp = G.last_stats()
        rs = pg.propagate_s(G, seeds, opts=opts, stream=sptr)
        sts = G.last_stats()
        pg.metrics(rp, g.n)
        return rp, rs, stp, sts

    # warm-up (also fixes the per-step work)
    for _ in range(args.warmup):
        rp, rs, stp, sts = step(opts_time)
    assert np.array_equal(rp.counts, rs.counts), "PROPAGATE-P and -S disagree"
    work_p = rp.seed_edge_traversals
    work_step = 2 * work_p
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, pull_ms, pull_launches, pull_b, post_ms, launches = [], 0.0, 0, 0.0, 0.0, 0
    p_ms, s_ms = [], []
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush, outside the timed events
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            rp = pg.propagate_p(G, seeds, opts=opts_time, stream=sptr)
            stp = G.last_stats()
            e1.record(stream)
            rs = pg.propagate_s(G, seeds, opts=opts_time, stream=sptr)
            sts = G.last_stats()
            pg.metrics(rp, g.n)
            e2.record(stream)
            e2.synchronize()
            times.append(e0.elapsed_time(e2))
            p_ms.append(e0.elapsed_time(e1))
            s_ms.append(e1.elapsed_time(e2))
            for st in (stp, sts):
                pull_ms += st["ms_pull"]
                pull_launches += st["pull_launches"]
                pull_b += pull_bytes(st)
                post_ms += st["ms_post"]
                launches += st["launches"]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.summary()
    total_ms = reduce_max(sum(times), world, dev)
    total_work = reduce_sum(float(work_step * args.steps), world, dev)
    value = total_work / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: graph upload, both
    # propagations, counts back to the host, metrics, graph freed
    h2d = g.row_ptr.nbytes + g.col.nbytes + 2 * seeds.nbytes
    d2h = rp.counts.nbytes + rp.m_active.nbytes + rs.counts.nbytes + rs.m_active.nbytes
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = pg.Graph.from_inputs(g, stream=sptr)
        r1 = pg.propagate_p(G2, seeds, opts=opts_run, stream=sptr)
        r2 = pg.propagate_s(G2, seeds, opts=opts_run, stream=sptr)
        pg.metrics(r1, g.n)
        G2.close()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    assert np.array_equal(r1.counts, rp.counts) and np.array_equal(r2.counts, rp.counts)
    e2e_total = reduce_max(sum(e2e_ms), world, dev)
    e2e_value = reduce_sum(float(work_step * len(e2e_ms)), world, dev) / (e2e_total / 1e3)

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (pull_b / max(pull_launches, 1)) / ((pull_ms / max(pull_launches, 1)) / 1e3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "pull_traffic.json")
    if os.path.exists(tpath):
        tr = json.load(open(tpath))
        if tr.get("workload") == args.workload and tr.get("kernel_hash") == kernel_hash():
            traffic = tr.get("bytes_per_launch")

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m, "s": s,
                   "rounds": rp.rounds, "seed_edge_traversals_per_step": work_step,
                   "l2": "flushed between steps (512 MB write); inputs also exceed L2",
                   "parallelism": f"replicas x{world} (independent seed samples)"},
        "parts": {"propagate_p_ms": statistics.mean(p_ms), "propagate_s_ms": statistics.mean(s_ms),
                  "propagate_p_seed_edges_per_s": work_p / (statistics.mean(p_ms) / 1e3),
                  "propagate_s_seed_edges_per_s": work_p / (statistics.mean(s_ms) / 1e3)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_pull", "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                     "pull_ms_per_launch": pull_ms / max(pull_launches, 1),
                     "pull_share_of_step": pull_ms / max(sum(times), 1e-9),
                     "post_share_of_step": post_ms / max(sum(times), 1e-9)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_total / len(e2e_ms)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, seeds, s, args.cpu_seeds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2301_06499_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:12]


def oracle_sample(g, seeds, k, steps=1):
    """Times the oracle (one FIFO BFS per seed, threads over seeds) on the
    first k seeds. Its work is the method-defined count of that k-seed
    problem, k * sum_t m_active(t), with m_active computed by the oracle from
    the sample's own distances (nothing comes from the GPU path)."""
    import oracle
    threads = os.cpu_count() or 1
    sample = np.ascontiguousarray(seeds[:k])
    hist, _, dmat = oracle.seed_histograms(g, sample, threads=threads, with_distances=True)
    work = int(k) * int(oracle.m_active(g, dmat, hist.shape[1], threads=threads).sum())
    del dmat
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.seed_histograms(g, sample, threads=threads)
        times.append(time.perf_counter() - t0)
    return work, times, threads


def cpu_baseline(g, seeds, s, k):
    work, times, threads = oracle_sample(g, seeds, k)
    dt = times[0]
    return {"value": work / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"oracle BFS from {k} of the {s} seeds on the same graph "
                      f"({dt:.2f} s wall on {threads} threads), credited that k-seed "
                      f"problem's k*sum_t m_active(t)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    spec, s, desc = WORKLOADS[args.workload]
    g = make_graph(spec)
    from paper_2301_06499_gb300 import inputs as I
    seeds = I.seeds(g.n, s, seed_stream(args.workload, 0))
    k = args.cpu_seeds
    oracle_sample(g, seeds, k, steps=args.warmup)
    work, times, threads = oracle_sample(g, seeds, k, steps=args.steps)
    value = work * len(times) / sum(times)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m, "s": s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"oracle BFS from {k} of the {s} seeds per step, credited "
                                   f"that k-seed problem's k*sum_t m_active(t)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat22_directed_s256")
    ap.add_argument("--cpu-seeds", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-launches", action="store_true",
                    help="launch every round kernel on the stream (no CUDA graph), e.g. under ncu")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
