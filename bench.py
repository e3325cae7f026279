"""Benchmark of the PROPAGATE hot path on GB300.

One step = PROPAGATE-P (Alg. 1) and PROPAGATE-S (Alg. 2) over the same seeds
on the benchmark workload, to fixpoint, through the C ABI, plus the Sec. 3
metrics from the counts. Work per step is the method-defined seed-edge
traversal count: each of the two runs solves the problem whose work is
sum_t s * m_active(t) (m_active from the PROPAGATE-P run).

Default workload: undirected R-MAT, scale 26 (67,108,864 nodes), edge factor
16, (a, b, c, d) = (.57, .19, .19, .05), RNG seed 2, symmetrised, duplicates
removed (~2.1 B arcs, int64 row pointers); s = 512 seeds (8 words, 64 bytes
per node), uniform without replacement (RNG seed 2): the stand-in for the
paper's largest in-memory graphs (Sec. 5, Table 1). --workload selects the
other shapes (see WORKLOADS), e.g. the directed R-MAT of scale 22 with
s = 256 (rmat22_directed_s256).

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
    # the same graph with its arc arrays in pinned host memory, read over the
    # CPU-GPU link (PG_HOST_CSR): the out-of-core configuration
    "rmat26_undirected_s512_hostcsr": (dict(kind="rmat", scale=26, ef=16, seed=2, directed=False,
                                            host_csr=True), 512,
                                       "undirected R-MAT scale 26, edge factor 16, s=512, arc "
                                       "arrays in host memory"),
    "rmat23_undirected_s512": (dict(kind="rmat", scale=23, ef=16, seed=2, directed=False), 512,
                               "undirected R-MAT scale 23, edge factor 16, s=512 (profiling "
                               "stand-in for scale 26)"),
    # the serving workload's widest requests: eps = 0.05 on n = 1e6 gives
    # s = ceil(ln n / eps^2) rounded to 64 = 5568 seeds (87 words per node)
    "er1e6_s5568": (dict(kind="er", n=1_000_000, d=16, seed=6), 5568,
                    "undirected ER n=1e6 avg degree 16, s=5568 (wide signatures)"),
    # exact mode: every node a seed (all-pairs distances), 1563 words per node
    "exact_er1e5": (dict(kind="er", n=100_000, d=8, seed=8), 100_000,
                    "undirected ER n=1e5 avg degree 8, s=n (exact all-pairs)"),
    "exact_er3e4": (dict(kind="er", n=30_000, d=8, seed=8), 30_000,
                    "undirected ER n=3e4 avg degree 8, s=n (exact all-pairs; profiling "
                    "stand-in for n=1e5)"),
}
# Batched workload: 512 graphs, n log-uniform in [1e3, 1e6], ER / R-MAT / grid
# with RNG seed 4, s per graph from eps in {0.1, 0.2} (see inputs.mix).
BATCH_WORKLOADS = {
    "mix512_batched": (512, 1e3, 1e6, 4),
    "mix64_batched": (64, 1e3, 1e5, 4),
}
# Serving workload: a resident pool of 64 graphs of the batched mix plus ER
# graphs uploaded while serving (n = 2e6 and 1e6); per request eps in
# {0.05, 0.1, 0.2} sets s = ceil(ln n / eps^2) rounded up to a multiple of 64.
SERVE_WORKLOADS = {
    "serve_mix64": dict(pool=64, n_lo=1e3, n_hi=1e6, seed=4,
                        uploads=((2_000_000, 8.0, 5), (1_000_000, 16.0, 6)),
                        rates=(200.0, 2000.0), duration=4.0, max_requests=1000, burst=600,
                        variants=4),
}
SEED_RNG = {"rmat22_directed_s256": 2, "er1e4_s64": 1, "grid4096_s128": 3,
            "rmat26_undirected_s512": 2, "rmat26_undirected_s512_hostcsr": 2,
            "rmat23_undirected_s512": 2, "er1e6_s5568": 7,
            "exact_er1e5": 9, "exact_er3e4": 9}


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
    per work item 16 B (item) + 8 B (row bounds) + 8 Wp B (own signature); per
    in-arc scanned 4 B (column index), plus 1/8 B (its changed bit) when bits
    are tested; per delta gathered 8 Wp B; per changed row 8 Wp B (signature
    write)."""
    w = 8.0 * st["words_per_row"]
    bit = 0.125 if st.get("test_changed") else 0.0
    return (st["items"] * (24.0 + w) + st["arcs_scanned"] * (4.0 + bit)
            + st["rows_gathered"] * w + st["changed_rows"] * w)


def round_bytes(st: dict, s: int, s_mode: bool) -> float:
    """Algorithmic bytes of a call's rounds by the method's own work counts:
    per active row (|A_t|, the rows a round revisits) 8 B of row bounds plus
    its signature read and written (2 s/8 B); per active in-arc (m_active(t))
    a 4 B column index plus the neighbour's s/8 B signature; per changed row
    (|F_t|) a 4 B frontier entry. PROPAGATE-S works in passes of 64 one-bit
    planes, so its unit signature is 64 bits (8 B) and its active rows and
    arcs are counted per pass."""
    sb = min(64, s) / 8.0 if s_mode else s / 8.0
    return (st["active_rows"] * (8.0 + 2.0 * sb) + st["m_active_total"] * (4.0 + sb)
            + st["changed_rows"] * 4.0)


def kernel_name(st: dict) -> str:
    """Name of the pull kernel instantiation a call used (words per gather,
    lanes per group, PROPAGATE-S passes as words), as ncu prints it."""
    wp, cw = st["words_per_row"], st["words_per_gather"]
    if st.get("dense_tma"):  # dense rounds by TMA gathers (sparse ones by k_pull)
        return f"k_pull_tma<{cw}, {1 if st.get('pass_words', 1) > 1 else 0}>"
    if cw == 0:  # the wide-row kernel: words per lane held in registers
        nw = 1 if wp <= 32 else 2 if wp <= 64 else 3 if wp <= 96 else 4 if wp <= 128 else 0
        return f"k_pull_wide<{nw}, {1 if st.get('pass_words', 1) > 1 else 0}>"
    return f"k_pull<{cw}, {st['group_lanes']}, {1 if st.get('pass_words', 1) > 1 else 0}>"


DEFAULT_WORKLOAD = "rmat26_undirected_s512"
# steps (and warm-ups) of the batched-vs-plain comparison the default line carries
BATCH_STEPS = 3
# seeds of the oracle's timed sample per workload (one BFS per host thread;
# the scale-26 graph takes seconds per BFS): default 64
CPU_SEEDS = {"rmat26_undirected_s512": 16, "rmat26_undirected_s512_hostcsr": 16}


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
    t_gen = time.perf_counter()
    g = make_graph(spec)
    gen_s = time.perf_counter() - t_gen  # host generation, outside every timing
    seeds = I.seeds(g.n, s, seed_stream(args.workload, rank))
    stream = torch.cuda.current_stream()
    sptr = __import__("ctypes").c_void_p(stream.cuda_stream)
    host_csr = bool(spec.get("host_csr", False))
    G = pg.Graph.from_inputs(g, stream=sptr, host_csr=host_csr)
    # schedule options: the library's autotuner picks them for this graph and
    # these seeds (untimed; counts are checked identical across candidates)
    tuned = None
    o_p, o_s = pg.options(), pg.options()
    if args.tune:
        t0 = time.perf_counter()
        o_p, rep_p = pg.autotune(G, seeds, max_trials=args.tune_trials, stream=sptr)
        o_s, rep_s = pg.autotune(G, seeds, max_trials=args.tune_trials, stream=sptr,
                                 algorithm="s")
        keys = ("direction", "dense_threshold", "group_lanes", "test_changed",
                "words_per_thread", "wide_rows", "passes_together", "pass_words")
        tuned = {"tune_s": time.perf_counter() - t0,
                 "p": {k: pg.options_dict(o_p)[k] for k in keys} | {"trials": rep_p["trials"]},
                 "s": {k: pg.options_dict(o_s)[k] for k in keys} | {"trials": rep_s["trials"]}}

    def with_(o, **kw):
        o2 = pg.options(**{k: getattr(o, k) for k, _ in o._fields_})
        for k, v in kw.items():
            setattr(o2, k, v)
        return o2

    opts_time_p, opts_time_s = with_(o_p, timing=1), with_(o_s, timing=1)
    plain = 0 if args.plain_launches else 1
    opts_run_p, opts_run_s = with_(o_p, use_graphs=plain), with_(o_s, use_graphs=plain)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        rp = pg.propagate_p(G, seeds, opts=opts_time_p, stream=sptr)
        stp = G.last_stats()
        rs = pg.propagate_s(G, seeds, opts=opts_time_s, stream=sptr)
        sts = G.last_stats()
        pg.metrics(rp, g.n)
        return rp, rs, stp, sts

    # warm-up (also fixes the per-step work)
    for _ in range(args.warmup):
        rp, rs, stp, sts = step()
    assert np.array_equal(rp.counts, rs.counts), "PROPAGATE-P and -S disagree"
    work_p = rp.seed_edge_traversals
    work_step = 2 * work_p
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, post_ms, launches = [], 0.0, 0
    per_kernel = {}  # pull kernel name -> [ms, launches, bytes]
    p_ms, s_ms = [], []
    with Clocks(torch.cuda.current_device()) as clk:
        # NVTX range of the timed steps: a launch-list capture selects it with
        # ncu --nvtx --nvtx-include bench_timed/
        torch.cuda.nvtx.range_push("bench_timed")
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush, outside the timed events
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            rp = pg.propagate_p(G, seeds, opts=opts_time_p, stream=sptr)
            stp = G.last_stats()
            e1.record(stream)
            rs = pg.propagate_s(G, seeds, opts=opts_time_s, stream=sptr)
            sts = G.last_stats()
            pg.metrics(rp, g.n)
            e2.record(stream)
            e2.synchronize()
            times.append(e0.elapsed_time(e2))
            p_ms.append(e0.elapsed_time(e1))
            s_ms.append(e1.elapsed_time(e2))
            for st, s_mode in ((stp, False), (sts, True)):
                k = per_kernel.setdefault(kernel_name(st), [0.0, 0, 0.0, 0.0, 0.0])
                k[0] += st["ms_pull"]
                k[1] += st["pull_launches"]
                k[2] += pull_bytes(st)
                k[3] += round_bytes(st, s, s_mode)
                k[4] += st["ms_post"]
                post_ms += st["ms_post"]
                launches += st["launches"]
        torch.cuda.nvtx.range_pop()
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
    # the user's CSR, held in pinned host memory (allocated outside the timing)
    rp_pinned = torch.from_numpy(np.array(g.row_ptr)).pin_memory().numpy()
    col_pinned = torch.from_numpy(np.array(g.col)).pin_memory().numpy()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, args.e2e_steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = pg.Graph.from_csr(rp_pinned, col_pinned, g.n, directed=g.directed, stream=sptr,
                               host_csr=host_csr)
        r1 = pg.propagate_p(G2, seeds, opts=opts_run_p, stream=sptr)
        r2 = pg.propagate_s(G2, seeds, opts=opts_run_s, stream=sptr)
        pg.metrics(r1, g.n)
        G2.close()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    assert np.array_equal(r1.counts, rp.counts) and np.array_equal(r2.counts, rp.counts)
    e2e_total = reduce_max(sum(e2e_ms), world, dev)
    e2e_value = reduce_sum(float(work_step * len(e2e_ms)), world, dev) / (e2e_total / 1e3)

    peak, peak_src = _peak()
    traffic_table, earlier = load_traffic(args.workload)

    def traffic_of(name):
        """DRAM bytes per launch of this pull kernel, from the stored capture
        of the same sources: the same instantiation, else one that differs
        only in lanes per sparse-round piece (the dense sweep, which moves
        almost all the bytes, is the same code)."""
        if name in traffic_table:
            return traffic_table[name]
        fam = name.split(",")[0] + "," + name.split(",")[-1]
        for k, v in traffic_table.items():
            if k.split(",")[0] + "," + k.split(",")[-1] == fam:
                return v
        return None

    def roofline_of(name):
        ms, nl, design, alg, post = per_kernel[name]
        nl = max(nl, 1)
        ach = (alg / nl) / ((ms / nl) / 1e3) / 1e9
        design_ach = (design / nl) / ((ms / nl) / 1e3) / 1e9
        tr_now = traffic_of(name)
        extra = {}
        if tr_now is None and name in earlier:
            extra["traffic_earlier_build"] = dict(
                earlier[name], note="ncu DRAM bytes per launch of an earlier build of this "
                                    "kernel's sources (profiles/pull_traffic.json); not a "
                                    "measurement of the kernel timed here")
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": tr_now, **extra, "kernel": name,
                "algorithmic_bytes_per_launch": alg / nl,
                "bytes_basis": "per round |A_t|(8+s/4) + m_active(t)(4+s/8) + |F_t|*4 "
                               "(s = 64 per pass for PROPAGATE-S), from the library's own "
                               "per-round counters, divided by this kernel's time",
                "ms_per_launch": ms / nl, "launches": nl,
                "share_of_step": ms / max(sum(times), 1e-9), "peak_source": peak_src,
                "round_frac": (alg / ((ms + post) / 1e3) / 1e9) / peak,
                "design_bytes_per_launch": design / nl, "design_frac": design_ach / peak}

    ranked = sorted(per_kernel, key=lambda k: -per_kernel[k][0])
    roofline = roofline_of(ranked[0])
    roofline["post_share_of_step"] = post_ms / max(sum(times), 1e-9)
    others = [roofline_of(k) for k in ranked[1:]]

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m, "s": s,
                   "rounds": rp.rounds, "seed_edge_traversals_per_step": work_step,
                   "l2": "flushed between steps (512 MB write); inputs also exceed L2",
                   "parallelism": f"replicas x{world} (independent seed samples)",
                   "graph_generation_s": round(gen_s, 3),
                   "options": tuned or "library defaults (--tune 0)"},
        "parts": {"propagate_p_ms": statistics.mean(p_ms), "propagate_s_ms": statistics.mean(s_ms),
                  "propagate_p_seed_edges_per_s": work_p / (statistics.mean(p_ms) / 1e3),
                  "propagate_s_seed_edges_per_s": work_p / (statistics.mean(s_ms) / 1e3),
                  "propagate_s_own_seed_edges_per_s":
                      sts["seed_edge_traversals"] / (statistics.mean(s_ms) / 1e3),
                  "propagate_s_own_work_note": "PROPAGATE-S's own per-pass work "
                      "(sum over its 64-plane passes of 64 * m_active), beside the "
                      "method-defined PROPAGATE-P work both runs are credited with",
                  "p_rounds": {"rounds": rp.rounds, "dense_rounds": stp["dense_rounds"],
                               "m_active_total": stp["m_active_total"],
                               "active_rows": stp["active_rows"],
                               "changed_rows": stp["changed_rows"]}},
        "roofline": roofline,
        "roofline_other_kernels": others,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_total / len(e2e_ms)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    # the same graph drawn and built on the device (pg_graph_generate),
    # outside every timing: its time beside the host generator's
    dev_gen = None
    if spec["kind"] in ("rmat", "er", "grid") and not host_csr:
        kw = ({"scale": spec["scale"], "edge_factor": spec["ef"], "directed": spec["directed"]}
              if spec["kind"] == "rmat" else
              {"n": spec["n"], "avg_degree": spec["d"]} if spec["kind"] == "er" else
              {"rows": spec["rows"], "cols": spec["cols"], "p_delete": spec["p"]})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gd = pg.Graph.generate(spec["kind"], spec["seed"], stream=sptr, **kw)
        torch.cuda.synchronize()
        dev_gen = {"seconds": round(time.perf_counter() - t0, 3),
                   "same_size": (Gd.n, Gd.m) == (g.n, g.m)}
        Gd.close()
        torch.cuda.empty_cache()
    out["config"]["device_generation"] = dev_gen
    if args.batched and args.workload == DEFAULT_WORKLOAD:
        # the metric's own comparison, batched vs plain, on the mixed workload
        # of 512 graphs (library default schedules, fewer steps than the
        # headline so that the whole run stays within minutes)
        G.close()
        torch.cuda.empty_cache()
        out["batched"] = measure_batch("mix512_batched", rank, world, dev, BATCH_STEPS,
                                       BATCH_STEPS, 0, args.tune_trials, 1, peak, peak_src)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, seeds, s, cpu_seeds(args))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_batch(workload, rank, world, dev, steps, warmup, tune, tune_trials, e2e_steps,
                  peak, peak_src):
    """Batched PROPAGATE-P over the mixed workload against the plain loop
    (one pg_propagate_p per graph on the same resident graphs), over the
    same graphs and seeds; every graph's counts must be identical both ways.
    Returns the batched and plain throughputs, the dominant kernel's
    roofline (a timed run of each width class), an end-to-end figure and an
    oracle baseline on a sample of the mix."""
    import ctypes
    import torch
    import paper_2301_06499_gb300 as pg
    from paper_2301_06499_gb300 import inputs as I

    count, n_lo, n_hi, seed = BATCH_WORKLOADS[workload]
    t0 = time.perf_counter()
    items = I.mix(count, n_lo, n_hi, seed + 1000 * rank)  # each rank its own replica
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    graphs = [pg.Graph.from_inputs(it.graph, stream=sptr) for it in items]
    batch = pg.Batch()
    for it in items:
        batch.add_inputs(it.graph, it.seeds)
    opts = pg.options()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def plain():
        res, work, launches = [], 0, 0
        for G, it in zip(graphs, items):
            res.append(pg.propagate_p(G, it.seeds, opts=opts, stream=sptr))
            st = G.last_stats()
            work += st["seed_edge_traversals"]
            launches += st["launches"]
        return res, work, launches

    def batched():
        batch.run(opts=None if tune else opts, stream=sptr)
        return batch.stats()

    t0 = time.perf_counter()
    batch.run(opts=opts, stream=sptr)  # packs the graphs (host union + upload), untimed
    pack_s = time.perf_counter() - t0
    tuned = None
    if tune:  # the autotuner picks each width class's schedule, untimed
        t0 = time.perf_counter()
        tuned = batch.tune(max_trials=tune_trials, stream=sptr)
        tuned["tune_s"] = time.perf_counter() - t0
        tuned["classes"] = [{"graphs": ng, "words_per_thread": o["words_per_thread"],
                             "group_lanes": o["group_lanes"],
                             "dense_threshold": round(o["dense_threshold"], 3),
                             "test_changed": o["test_changed"]}
                            for ng, o in batch.group_options()]
    for _ in range(warmup):
        res_p, work, plain_launches = plain()
        bst = batched()
    mact_same = 0  # graphs whose own m_active in the batch equals the plain run's
    for k, r in enumerate(res_p):
        rb = batch.result(k)
        assert rb.rounds == r.rounds and np.array_equal(rb.counts, r.counts), items[k].graph.name
        mact_same += int(np.array_equal(rb.m_active, r.m_active))
    assert bst["seed_edge_traversals"] == work, (bst["seed_edge_traversals"], work)

    def timed(fn):
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        b_ms = timed(batched)
        p_ms = timed(plain)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    b_total = reduce_max(sum(b_ms), world, dev)
    p_total = reduce_max(sum(p_ms), world, dev)
    total_work = reduce_sum(float(work * steps), world, dev)
    value = total_work / (b_total / 1e3)
    plain_value = total_work / (p_total / 1e3)

    # the dominant pull kernel of the batched run: one more run with
    # per-kernel events (plain launches, library default schedule), per
    # group, the groups one after another so that each kernel time is its own
    batch.set_streams(1)
    batch.run(opts=pg.options(timing=1), stream=sptr)
    batch.set_streams(4)
    classes = []
    members = [ng for ng, _ in batch.group_options()]
    for gi, st in enumerate(batch.group_stats()):
        s_cls = 64 * st["words_per_row"]
        classes.append({"kernel": kernel_name(st), "s": s_cls, "graphs": members[gi],
                        "ms_pull": st["ms_pull"],
                        "pull_launches": st["pull_launches"], "ms_post": st["ms_post"],
                        "bytes": round_bytes(st, s_cls, False)})
    roofline = None
    timed_classes = [c for c in classes if c["pull_launches"] > 0 and c["ms_pull"] > 0]
    if timed_classes:
        top = max(timed_classes, key=lambda c: c["ms_pull"])
        ach = top["bytes"] / (top["ms_pull"] / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": None, "kernel": top["kernel"],
                    "width_class_s": top["s"],
                    "algorithmic_bytes_per_launch": top["bytes"] / top["pull_launches"],
                    "ms_per_launch": top["ms_pull"] / top["pull_launches"],
                    "launches": top["pull_launches"], "peak_source": peak_src,
                    "bytes_basis": "per round |A_t|(8+s/4) + m_active(t)(4+s/8) + |F_t|*4 "
                                   "over the group (a width class's packed union, or one "
                                   "large graph run alone; s = the class's seeds per graph), "
                                   "divided by its pull kernel's time",
                    "note": "a run with per-launch events (plain launches, library default "
                            "schedule, groups one after another) after the timed steps, "
                            "which run four groups at once"}

    # end to end with host buffers: pack, upload, run, read every result back
    h2d = sum(it.graph.row_ptr.nbytes + it.graph.col.nbytes + it.seeds.nbytes for it in items)
    d2h = sum(r.counts.nbytes for r in res_p)
    e2e_ms = []
    for _ in range(max(1, min(steps, e2e_steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with pg.Batch() as b2:
            for it in items:
                b2.add_inputs(it.graph, it.seeds)
            b2.run(opts=opts, stream=sptr)
            out = [b2.result(k) for k in range(len(items))]
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    assert all(np.array_equal(o.counts, r.counts) for o, r in zip(out, res_p))
    e2e_total = reduce_max(sum(e2e_ms), world, dev)
    e2e_value = reduce_sum(float(work * len(e2e_ms)), world, dev) / (e2e_total / 1e3)

    # the oracle on a sample of the mix: its first graphs, 8 seeds each
    cpu = None
    if rank == 0:
        import oracle
        wk, tt, nk = 0, 0.0, 0
        for it in items:
            if tt > 10.0:
                break
            w1, t1, threads = oracle_sample(it.graph, it.seeds, min(8, it.s), steps=1)
            wk += w1
            tt += min(t1)
            nk += 1
        cpu = {"value": wk / tt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"oracle BFS from 8 seeds of each of the mix's first {nk} graphs "
                         f"({tt:.2f} s), credited each sample's own k*sum_t m_active(t)"}

    widths = sorted({(it.s + 63) // 64 for it in items})
    out = {
        "value": value, "ms_per_step": b_total / steps,
        "plain": {"value": plain_value, "ms_per_step": p_total / steps,
                  "gpu_launches": int(plain_launches)},
        "batched_over_plain": plain_value and value / plain_value,
        "counts_identical": True,
        "m_active_identical_graphs": f"{mact_same} of {len(items)}",
        "config": {"workload": workload,
                   "description": f"{count} graphs, n log-uniform in [{n_lo:g}, {n_hi:g}], "
                                  f"ER/R-MAT/grid (RNG {seed}), s from eps in {{0.1, 0.2}}",
                   "sum_n": int(sum(it.graph.n for it in items)),
                   "sum_m": int(sum(it.graph.m for it in items)),
                   "sum_s": int(sum(it.s for it in items)), "signature_words": widths,
                   "groups": bst["groups"], "batched_rounds": bst["sweeps"],
                   "seed_edge_traversals_per_step": int(work),
                   "generate_s": gen_s, "pack_s": pack_s, "steps": steps, "warmup": warmup,
                   "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world} (independent mixes)"},
        "autotune": tuned,
        "groups": classes,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_total / len(e2e_ms)},
        "gpu_launches": int(bst["launches"]),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    batch.close()
    for G in graphs:
        G.close()
    return out


def _peak():
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    src = ("measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
           else "fallback 6.8 TB/s (profiling recipe)")
    return peak, src


def run_batch(args):
    """The mixed workload alone: batched seed-edge traversals/s, with the
    plain loop's beside it (see measure_batch)."""
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    peak, peak_src = _peak()
    r = measure_batch(args.workload, rank, world, dev, args.steps, args.warmup, args.tune,
                      args.tune_trials, args.e2e_steps, peak, peak_src)
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": r["config"], "plain": r["plain"],
        "batched_over_plain": r["batched_over_plain"], "counts_identical": r["counts_identical"],
        "m_active_identical_graphs": r["m_active_identical_graphs"], "autotune": r["autotune"],
        "groups": r["groups"], "roofline": r["roofline"], "e2e": r["e2e"],
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        "cpu_baseline": r["cpu_baseline"],
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _serve_requests(count, n_graphs, seed, variants, upload_at=None):
    """count requests: (graph index, eps, variant), graph uniform over the
    graphs available (uploaded graphs join at their index in upload_at)."""
    from paper_2301_06499_gb300 import inputs as I
    out = []
    for k in range(count):
        avail = n_graphs if upload_at is None else upload_at(k)
        gi = int(I.rand(seed, 40, k) % avail)
        eps = (0.05, 0.1, 0.2)[I.rand(seed, 41, k) % 3]
        v = int(I.rand(seed, 42, k) % variants)
        out.append((gi, eps, v))
    return out


def run_serve(args):
    """Serving loop (pg_server) against the plain one-request-at-a-time loop
    (pg_propagate_p per request on resident graphs) over the same request
    sequence; then open-loop Poisson arrivals with p50/p99 latency. Every
    served answer is checked against the request run alone. Wall-clock
    timing (the work spans several streams and threads), bracketed by device
    synchronisation."""
    import ctypes
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

    W = SERVE_WORKLOADS[args.workload]
    t0 = time.perf_counter()
    graphs = [it.graph for it in I.mix(W["pool"], W["n_lo"], W["n_hi"], W["seed"] + 1000 * rank)]
    uploads = [I.er(n, d, sd + 1000 * rank) for n, d, sd in W["uploads"]]
    gen_s = time.perf_counter() - t0
    allg = graphs + uploads
    V = W["variants"]
    seed_cache = {}

    def seeds_of(gi, eps, v):
        key = (gi, eps, v)
        if key not in seed_cache:
            n = allg[gi].n
            s = min(n, I.s_rounded_64(n, eps))
            seed_cache[key] = I.seeds(n, s, 7_000_003 * gi + 1009 * int(eps * 100) + v)
        return seed_cache[key]

    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    handles = [pg.Graph.from_inputs(g, stream=sptr) for g in allg]
    alone = {}  # (gi, eps, v) -> (counts, rounds, work)

    def run_alone(key):
        gi, eps, v = key
        r = pg.propagate_p(handles[gi], seeds_of(*key), stream=sptr)
        w = handles[gi].last_stats()["seed_edge_traversals"]
        return r, w

    # closed loop: the same `burst` requests, plain loop vs server
    burst = _serve_requests(W["burst"], len(allg), W["seed"] + 7, V)
    for key in set(burst):
        r, w = run_alone(key)
        alone[key] = (r.counts, r.rounds, w)
    for key in burst[:8]:  # warm-up of the plain loop
        run_alone(key)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_work = 0
    for key in burst:
        _, w = run_alone(key)
        plain_work += w
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0

    srv = pg.Server(slots=args.slots, cross_graph=bool(args.cross_graph))
    gids = [srv.add_inputs(g) for g in graphs]  # the uploads join while serving
    upload_s = []

    def served(reqs, arrivals=None, uploads_at=()):
        """Submits reqs (at the given arrival offsets, else at once) from a
        producer thread, which also registers uploads[j] just before request
        uploads_at[j]; returns per-request latencies (ms), mismatches, wall s."""
        import threading
        rids = [None] * len(reqs)
        sem = threading.Semaphore(0)
        start = time.perf_counter()

        def produce():
            for k, key in enumerate(reqs):
                if arrivals is not None:
                    d = start + arrivals[k] - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                for j, at in enumerate(uploads_at):
                    if at == k:
                        t = time.perf_counter()
                        gids.append(srv.add_inputs(uploads[j]))
                        upload_s.append(time.perf_counter() - t)
                rids[k] = srv.submit(gids[key[0]], seeds_of(*key))
                sem.release()

        th = threading.Thread(target=produce)
        th.start()
        lat, bad = [], 0
        for k, key in enumerate(reqs):
            sem.acquire()
            res, info = srv.result(rids[k])
            lat.append((info["done_ns"] - info["submit_ns"]) / 1e6)
            c, T, _ = alone[key]
            bad += int(res.rounds != T or not np.array_equal(res.counts, c))
        th.join()
        torch.cuda.synchronize()
        return lat, bad, time.perf_counter() - start

    def ensure_alone(reqs):
        for key in set(reqs):
            if key not in alone:
                r, w = run_alone(key)
                alone[key] = (r.counts, r.rounds, w)

    def open_loop_run(rate, uploads_at=(), count=None):
        count = count or min(int(rate * W["duration"]), W["max_requests"])
        rng = np.random.default_rng(W["seed"] + int(rate * 1000))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
        first = len(graphs)

        def avail(k):  # graphs registered by the time request k is submitted
            return first + sum(1 for at in uploads_at if at <= k) if uploads_at else len(allg)

        reqs = _serve_requests(count, len(allg), W["seed"] + int(rate * 1000), V,
                               upload_at=avail)
        ensure_alone(reqs)
        lat, bad, wall = served(reqs, arrivals, uploads_at)
        assert bad == 0, f"{bad} served answers differ from the request alone"
        rwork = sum(alone[k][2] for k in reqs)
        return {"offered_req_per_s": rate, "requests": count, "wall_s": wall,
                "achieved_req_per_s": count / wall,
                "seed_edge_traversals_per_s": rwork / wall,
                "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(max(lat))}

    warm = [k for k in burst if k[0] < len(graphs)][:16]
    served(warm)  # warm-up: views, workspaces, captured loops
    open_loop = []
    with Clocks(torch.cuda.current_device()) as clk:
        n0 = min(int(W["rates"][0] * W["duration"]), W["max_requests"])
        open_loop.append(open_loop_run(W["rates"][0], uploads_at=(n0 // 3, 2 * n0 // 3)))
        st0 = srv.stats()
        lat_b, bad_b, served_s = served(burst)
        st1 = srv.stats()
        assert bad_b == 0, f"{bad_b} served answers differ from the request alone"
        work = sum(alone[k][2] for k in burst)
        assert work == plain_work
        value = work / served_s
        plain_value = work / plain_s
        # capacity: the burst's completion rate; latency below and at it, so
        # that p50/p99 are not queueing alone
        capacity = len(burst) / served_s
        for frac in (0.5, 0.9):
            rate = frac * capacity
            r = open_loop_run(rate, count=int(max(60, min(300, rate * 20))))
            r["fraction_of_capacity"] = frac
            open_loop.append(r)
        for rate in W["rates"][1:]:
            open_loop.append(open_loop_run(rate))
    stats = srv.stats()
    srv.close()

    h2d = sum(seeds_of(*k).nbytes for k in burst)
    d2h = sum(alone[k][0].nbytes for k in burst)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": served_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "description": f"pool of {W['pool']} mixed graphs (n log-uniform "
                                  f"[{W['n_lo']:g}, {W['n_hi']:g}]) + uploaded ER "
                                  f"{[u[0] for u in W['uploads']]}; eps in {{0.05, 0.1, 0.2}}",
                   "burst_requests": len(burst), "slots": args.slots,
                   "cross_graph": bool(args.cross_graph),
                   "distinct_requests": len(alone), "generate_s": gen_s,
                   "timing": "wall clock between device synchronisations",
                   "parallelism": f"replicas x{world}"},
        "plain": {"value": plain_value, "ms_per_step": plain_s * 1e3},
        "served_over_plain": value / plain_value,
        "capacity_req_per_s": capacity,
        "burst_latency_ms": {"p50": float(np.percentile(lat_b, 50)),
                             "p99": float(np.percentile(lat_b, 99))},
        "burst_propagations": st1["propagations"] - st0["propagations"],
        "open_loop": open_loop,
        "upload_while_serving_s": upload_s,
        "server": {k: stats[k] for k in ("peak_bytes", "budget_bytes", "resident_bytes",
                                          "completed", "propagations")},
        "roofline": None,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": served_s * 1e3},
        "gpu_launches": int(st1["gpu_launches"] - st0["gpu_launches"]),
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    for G in handles:
        G.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def load_traffic(workload: str, path: str | None = None):
    """The stored ncu DRAM bytes per pull launch of `workload`
    (profiles/pull_traffic.json): ({kernel: bytes} for kernels whose sources
    still hash as captured, {kernel: {...}} for captures of an earlier build
    of a kernel's sources, reported as context only)."""
    path = path or os.path.join(ROOT, "profiles", "pull_traffic.json")
    table, earlier = {}, {}
    if not os.path.exists(path):
        return table, earlier
    tr = json.load(open(path))
    if tr.get("workload") != workload:
        return table, earlier
    hashes = tr.get("kernel_hash", {})
    hashes = hashes if isinstance(hashes, dict) else {}
    for k, v in tr.get("bytes_per_launch", {}).items():
        if hashes.get(k) == kernel_hash(k):
            table[k] = v
        else:
            earlier[k] = {"bytes_per_launch": v, "sources_hash": hashes.get(k),
                          "current_sources_hash": kernel_hash(k)}
    return table, earlier


def kernel_hash(kernel: str) -> str:
    """Hash of the sources that define one pull kernel instantiation (its
    device code and the parameter block): a stored DRAM-traffic figure
    applies only to the kernel it was captured from."""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2301_06499_gb300", "csrc")
    if kernel.startswith("k_pull_wide"):
        own = "pull_wide.cu"
    elif kernel.startswith("k_pull_tma"):
        own = "pull_tma.cu"
    else:
        m = re.match(r"k_pull<(\d+)", kernel)
        own = f"pull_cw{m.group(1)}.cu" if m else ""
    for name in ("common.cuh", "kernels.cuh", "push.cu", own):
        path = os.path.join(csrc, name)
        if name and os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:12]


def cpu_seeds(args) -> int:
    return args.cpu_seeds or CPU_SEEDS.get(args.workload, 64)


# distance capacity of the oracle's histograms (R-MAT and ER eccentricities are
# tens; the 4096^2 grid's is ~8,000): the oracle reports an overflow
HIST_CAP = 1 << 15


def oracle_sample(g, seeds, k, steps=1, threads=None, budget_s=None):
    """Times the oracle (one FIFO BFS per seed, threads over seeds) on the
    first k seeds: the run that also records distances, then up to `steps`
    more runs while the total stays within budget_s seconds. Returns the
    work, every run's time (the first is the distance-recording run) and the
    threads. The work is the method-defined count of that k-seed problem,
    k * sum_t m_active(t), with m_active computed by the oracle from the
    sample's own distances (nothing comes from the GPU path)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    sample = np.ascontiguousarray(seeds[:k])
    t0 = time.perf_counter()
    hist, _, dmat = oracle.seed_histograms(g, sample, cap=min(g.n, HIST_CAP), threads=threads,
                                           with_distances=True)
    times = [time.perf_counter() - t0]
    work = int(k) * int(oracle.m_active(g, dmat, hist.shape[1], threads=threads).sum())
    del dmat
    for _ in range(steps):
        if budget_s is not None and sum(times) > budget_s:
            break
        t0 = time.perf_counter()
        oracle.seed_histograms(g, sample, cap=min(g.n, HIST_CAP), threads=threads)
        times.append(time.perf_counter() - t0)
    return work, times, threads


# wall-clock bound of the reference arm's oracle runs
REF_BUDGET_S = 240.0
# one host sweep of Alg. 1 reads every arc: beyond this many the bench skips it
ALG1_MAX_ARCS = 1 << 28


def cpu_baseline(g, seeds, s, k):
    """The oracle's BFS on all host cores (and on one, over fewer seeds), and
    the paper's own method, Alg. 1 swept on the host (oracle.propagate_p), on
    the same k-seed sample and credited the same work."""
    import oracle
    work, times, threads = oracle_sample(g, seeds, k, steps=5, budget_s=15.0)
    dt = min(times[1:] or times)
    how = (f"best of {len(times) - 1} after a warm-up" if len(times) > 1 else
           "one run (it also records the distances the work count needs; a run takes "
           "longer than the bench's CPU budget)")
    out = {"value": work / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"oracle BFS from {k} of the {s} seeds on the same graph, {how} "
                     f"({dt:.2f} s wall on {threads} threads, the oracle's own CSR check and "
                     f"transpose included), credited that k-seed problem's k*sum_t m_active(t)"}
    if g.m <= ALG1_MAX_ARCS:
        k1 = min(4, k)
        work1, times1, _ = oracle_sample(g, seeds, k1, steps=5, threads=1, budget_s=10.0)
        t1 = min(times1[1:] or times1)
        out["value_1_thread"] = work1 / t1
        out["sample_1_thread"] = f"oracle BFS from {k1} seeds on one thread ({t1:.2f} s)"
    if g.m > ALG1_MAX_ARCS:
        out["alg1_host"] = {"skipped": f"{g.m} arcs: a host sweep per round exceeds the "
                                       f"bench's CPU budget"}
        return out
    sample = np.ascontiguousarray(seeds[:k])
    oracle.propagate_p(g, sample, threads=threads)  # warm-up
    ta = []
    for _ in range(5):  # best of five, within the CPU budget
        t0 = time.perf_counter()
        oracle.propagate_p(g, sample, threads=threads)
        ta.append(time.perf_counter() - t0)
        if sum(ta) > 15.0:
            break
    out["alg1_host"] = {"value": work / min(ta), "unit": UNIT, "cores": threads,
                        "kind": "Alg. 1 on the host (oracle.propagate_p)",
                        "sample": f"{k} of the {s} seeds as {k}-bit signatures, best of "
                                  f"{len(ta)} after a warm-up ({min(ta):.2f} s), credited "
                                  f"the same work as the BFS sample"}
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    spec, s, desc = WORKLOADS[args.workload]
    g = make_graph(spec)
    from paper_2301_06499_gb300 import inputs as I
    seeds = I.seeds(g.n, s, seed_stream(args.workload, 0))
    k = cpu_seeds(args)
    # run 0 records distances (for the work count) and is a warm-up; runs
    # 1..W-1 are warm-ups; the next K are timed, within REF_BUDGET_S seconds
    work, times, threads = oracle_sample(g, seeds, k, steps=args.warmup - 1 + args.steps,
                                         budget_s=REF_BUDGET_S)
    warm = min(args.warmup, len(times) - 1)
    timed = times[warm:]
    value = work * len(timed) / sum(timed)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": len(timed), "warmup": warm,
        "ms_per_step": 1e3 * sum(timed) / len(timed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m, "s": s,
                   "steps_requested": args.steps, "warmup_requested": args.warmup,
                   "time_bound": f"runs stop once {REF_BUDGET_S:.0f} s are spent (one oracle "
                                 f"run over the scale-26 graph takes about a minute); at least "
                                 f"one run is timed"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"oracle BFS from {k} of the {s} seeds per step (the "
                                   f"oracle's own CSR check and transpose included), credited "
                                   f"that k-seed problem's k*sum_t m_active(t)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def profile_run(args):
    """Builds the workload, tunes it like the bench, and calls PROPAGATE-P or
    -S twice with plain launches and per-launch events (no CUDA graph): the
    program profiled by ncu. The second call runs like a timed bench call
    (the first call's round count is its hint) inside the NVTX range
    "bench_call", which captures select; prints each call's launches."""
    import torch
    torch.cuda.set_device(0)
    import paper_2301_06499_gb300 as pg
    from paper_2301_06499_gb300 import inputs as I
    spec, s, _ = WORKLOADS[args.workload]
    g = make_graph(spec)
    seeds = I.seeds(g.n, s, seed_stream(args.workload, 0))
    G = pg.Graph.from_inputs(g)
    fn = pg.propagate_p if args.profile_run == "p" else pg.propagate_s
    o = pg.options()
    if args.tune:  # the schedule the bench times
        o, _ = pg.autotune(G, seeds, max_trials=args.tune_trials, algorithm=args.profile_run)
    o.use_graphs, o.timing = 0, 1
    calls = []
    for k in range(2):
        if k == 1:  # the call a capture selects: ncu --nvtx --nvtx-include "bench_call/"
            torch.cuda.nvtx.range_push("bench_call")
        res = fn(G, seeds, opts=o)
        if k == 1:
            torch.cuda.nvtx.range_pop()
        st = G.last_stats()
        calls.append({"pull_launches": st["pull_launches"], "post_launches": st["post_launches"],
                      "rounds": res.rounds, "ms_pull": st["ms_pull"]})
    print(json.dumps({"workload": args.workload, "options": pg.options_dict(o), "calls": calls}))


def write_traffic(workload: str, csvs: list, out_path: str | None = None) -> dict:
    """profiles/pull_traffic.json from ncu CSV captures of the pull kernels
    (dram__bytes_read.sum and dram__bytes_write.sum): mean bytes per launch
    of each kernel, with the hash of the sources it was built from."""
    import ncu_summary
    per, push = {}, {}
    for path in csvs:
        tot = ncu_summary.traffic_totals(path)
        pushed = sum(b for k, (b, _) in tot.items() if k.startswith("k_push"))
        for k, (b, nl) in tot.items():
            if k.startswith("k_push"):
                push[k] = b / nl
            elif k.startswith("k_pull"):
                # a round's pull time includes its push kernel: so do its bytes
                per[k] = (b + pushed) / nl
    out = {"workload": workload,
           "kernel_hash": {k: kernel_hash(k) for k in per},
           "bytes_per_launch": per,
           "push_bytes_per_launch": push,
           "commands": [
               f"python bench.py --profile-run p --workload {workload}",
               "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
               "--nvtx --nvtx-include bench_call/ --clock-control none -k regex:'k_pu(ll|sh)' --csv "
               f"--log-file traffic_p.csv python bench.py --profile-run p --workload {workload}",
               "(the same two lines with --profile-run s -> traffic_s.csv)",
               "python bench.py --workload " + workload +
               " --write-traffic traffic_p.csv traffic_s.csv"],
           "note": "dram__bytes_read.sum + dram__bytes_write.sum of the pull launches, and of "
                   "the push launches that follow them in push rounds, over the call the bench "
                   "times (NVTX range bench_call, autotuned schedule), per pull launch (the "
                   "library's pull time of a round spans both kernels); a kernel's figure "
                   "applies while the hash of its sources (common.cuh, kernels.cuh, push.cu "
                   "and its pull_*.cu) is unchanged"}
    with open(out_path or os.path.join(ROOT, "profiles", "pull_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(per))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) +
                    sorted(SERVE_WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--slots", type=int, default=4, help="server slots (serving workload)")
    ap.add_argument("--cross-graph", type=int, default=1,
                    help="server: 1 = merge requests across graphs of one width as a union")
    ap.add_argument("--tune", type=int, default=1,
                    help="1 = let the autotuner pick the schedule options before timing")
    ap.add_argument("--tune-trials", type=int, default=16)
    ap.add_argument("--cpu-seeds", type=int, default=0,
                    help="seeds of the oracle's timed sample (0 = per workload: 16 on the "
                         "scale-26 graph, else 64)")
    ap.add_argument("--batched", type=int, default=1,
                    help="1 = the default workload's line also carries the batched-vs-plain "
                         "comparison on the 512-graph mix (key 'batched')")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="end-to-end steps (graph upload + both runs + metrics), at most --steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-launches", action="store_true",
                    help="launch every round kernel on the stream (no CUDA graph), e.g. under ncu")
    ap.add_argument("--profile-run", choices=["p", "s"],
                    help="only build the workload and run PROPAGATE-P/-S twice (for ncu)")
    ap.add_argument("--write-traffic", nargs="+", metavar="CSV",
                    help="write profiles/pull_traffic.json from ncu captures of the pull kernels")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.write_traffic:
        write_traffic(args.workload, args.write_traffic)
    elif args.profile_run:
        profile_run(args)
    elif args.workload in SERVE_WORKLOADS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the "
                              "single-graph workloads; run it without --workload"}))
        else:
            run_serve(args)
    elif args.workload in BATCH_WORKLOADS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the "
                              "single-graph workloads; run it without --workload"}))
        else:
            run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
