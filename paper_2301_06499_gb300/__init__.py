"""PROPAGATE on GB300: exact per-seed ball sizes by Boolean seed propagation.

Python binding of the C ABI in ``include/propagate.h`` (names kept). It only
marshals arguments: graphs, seeds and result buffers go to the CUDA library,
which runs every step (seed set-up, pull rounds, per-seed counts, frontier,
fixpoint test). PyTorch, when present, only supplies device memory and the
current CUDA stream.

    g = Graph.from_csr(row_ptr, col, directed=True)       # CSR over in-edges
    res = propagate_p(g, seeds)                            # Algorithm 1
    res_s = propagate_s(g, seeds)                          # Algorithm 2
    m = metrics(res, g.n)                                  # Sec. 3 metrics

    b = Batch(); i = b.add(row_ptr, col, seeds); b.run()   # many graphs at once
    res_i = b.result(i)

    srv = Server(slots=4); gid = srv.add_graph(row_ptr, col)  # serving loop
    rid = srv.submit(gid, seeds); res = srv.result(rid)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _abi
from ._abi import (PG_DIR_AUTO, PG_DIR_DENSE, PG_DIR_SPARSE, PropagateError)

__all__ = ["Graph", "Result", "Batch", "Server", "autotune", "options_dict", "progressive",
           "propagate_p", "propagate_s", "metrics", "options",
           "PropagateError", "PG_DIR_AUTO", "PG_DIR_DENSE", "PG_DIR_SPARSE", "library_path"]


def library_path() -> str:
    from . import build
    return build.LIB


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def options(**kw) -> _abi.Options:
    """pg_options with the library defaults, overridden by keyword."""
    o = _abi.Options()
    _abi.lib().pg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def options_dict(o: _abi.Options) -> dict:
    return {f: getattr(o, f) for f, _ in _abi.Options._fields_}


class Graph:
    """Device-resident CSR over in-edges (pg_graph)."""

    def __init__(self, handle, n: int, m: int, keep=None):
        self._h = handle
        self.n = n
        self.m = m
        self._keep = keep  # borrowed device tensors must outlive the handle

    @classmethod
    def from_csr(cls, row_ptr, col, n: int | None = None, directed: bool = True,
                 stream=None, reverse: bool = False, relabel: bool | None = None,
                 host_csr: bool = False) -> "Graph":
        """row_ptr int64[n+1] and col int32[m] as numpy arrays (copied from the
        host) or CUDA torch tensors (used in place). reverse=True counts balls
        grown backward (nodes reaching each seed; PG_REVERSE). relabel: True =
        PG_RELABEL, False = PG_KEEP_ORDER, None = the library's default."""
        rev = _abi.PG_REVERSE if reverse else 0
        if relabel is not None:
            rev |= _abi.PG_RELABEL if relabel else _abi.PG_KEEP_ORDER
        if host_csr:  # arc arrays in pinned host memory (PG_HOST_CSR)
            rev |= _abi.PG_HOST_CSR
        L = _abi.lib()
        h = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        keep = None
        if hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda and not host_csr:
            import torch
            rp = row_ptr.to(torch.int64).contiguous()
            cl = col.to(torch.int32).contiguous()
            n = rp.numel() - 1 if n is None else n
            m = cl.numel()
            flags = _abi.PG_DEVICE_PTRS | _abi.PG_BORROW | rev
            rc = L.pg_graph_from_csr(rp.data_ptr(), cl.data_ptr() if m else None, n, m,
                                     int(directed), flags, st, ctypes.byref(h))
            keep = (rp, cl)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            n = rp.size - 1 if n is None else n
            m = cl.size
            rc = L.pg_graph_from_csr(rp.ctypes.data, cl.ctypes.data if m else None, n, m,
                                     int(directed), rev, st, ctypes.byref(h))
        _abi.check(rc, "pg_graph_from_csr")
        return cls(h, int(n), int(m), keep)

    @classmethod
    def from_inputs(cls, g, stream=None, reverse: bool = False,
                    relabel: bool | None = None, host_csr: bool = False) -> "Graph":
        """From a generated graph (``inputs.Graph``) held in host memory."""
        return cls.from_csr(g.row_ptr, g.col, g.n, directed=g.directed, stream=stream,
                            reverse=reverse, relabel=relabel, host_csr=host_csr)

    @classmethod
    def generate(cls, kind: str, seed: int, stream=None, reverse: bool = False,
                 relabel: bool | None = None, **kw) -> "Graph":
        """pg_graph_generate: a seeded synthetic graph drawn and built on the
        device. kind "er" (n, avg_degree), "rmat" (scale, edge_factor,
        directed, a=.57, b=.19, c=.19) or "grid" (rows, cols, p_delete)."""
        gen = _abi.Generator()
        gen.seed = int(seed)
        if kind == "er":
            gen.kind, gen.n, gen.avg_degree = _abi.PG_GEN_ER, int(kw["n"]), float(kw["avg_degree"])
        elif kind == "rmat":
            gen.kind, gen.scale = _abi.PG_GEN_RMAT, int(kw["scale"])
            gen.edge_factor, gen.directed = float(kw["edge_factor"]), int(bool(kw["directed"]))
            gen.a, gen.b, gen.c = (float(kw.get("a", 0.57)), float(kw.get("b", 0.19)),
                                   float(kw.get("c", 0.19)))
        elif kind == "grid":
            gen.kind, gen.rows, gen.cols = _abi.PG_GEN_GRID, int(kw["rows"]), int(kw["cols"])
            gen.p_delete = float(kw["p_delete"])
        else:
            raise ValueError(f"unknown generator {kind!r}")
        flags = _abi.PG_REVERSE if reverse else 0
        if relabel is not None:
            flags |= _abi.PG_RELABEL if relabel else _abi.PG_KEEP_ORDER
        h = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _abi.check(_abi.lib().pg_graph_generate(ctypes.byref(gen), flags, st, ctypes.byref(h)),
                   "pg_graph_generate")
        n, m = ctypes.c_int64(), ctypes.c_int64()
        _abi.check(_abi.lib().pg_graph_info(h, ctypes.byref(n), ctypes.byref(m)), "pg_graph_info")
        return cls(h, int(n.value), int(m.value))

    def csr(self, stream=None):
        """pg_graph_copy_csr: (row_ptr, col) as the kernels read them (the
        internal ids of a relabelled graph)."""
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.m, 1), dtype=np.int32)
        st = stream if stream is not None else _current_stream()
        _abi.check(_abi.lib().pg_graph_copy_csr(self._h, rp.ctypes.data, col.ctypes.data, st),
                   "pg_graph_copy_csr")
        return rp, col[:self.m]

    @property
    def relabelled(self) -> bool:
        r = ctypes.c_int32()
        _abi.check(_abi.lib().pg_graph_is_relabelled(self._h, ctypes.byref(r)),
                   "pg_graph_is_relabelled")
        return bool(r.value)

    def rounds_bound(self) -> int:
        r = ctypes.c_int32()
        _abi.check(_abi.lib().pg_query_rounds_bound(self._h, ctypes.byref(r)),
                   "pg_query_rounds_bound")
        return int(r.value)

    def last_stats(self) -> dict:
        st = _abi.Stats()
        _abi.check(_abi.lib().pg_last_stats(self._h, ctypes.byref(st)), "pg_last_stats")
        return {f: getattr(st, f) for f, _ in _abi.Stats._fields_}

    def close(self):
        if self._h:
            _abi.lib().pg_graph_free(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


@dataclass
class Result:
    """Output of one propagation.

    counts   uint32[T+1, s]: counts[t, i] = nodes at distance exactly t from
             seed i (row 0 all ones); T = rounds = Delta_LB of Alg. 1.
    m_active uint64[T+2]: arcs the round-t sweep revisits (entry T+1 is the
             final sweep that found no change).
    """
    rounds: int
    counts: np.ndarray
    m_active: np.ndarray
    s: int
    n: int

    @property
    def seed_edge_traversals(self) -> int:
        """sum_t s * m_active(t): the work measure of the benchmark."""
        return int(self.s) * int(self.m_active.astype(np.uint64).sum())


def _run(fn, what, g: Graph, seeds, max_rounds, opts, stream) -> Result:
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    s = int(seeds.size)
    st = stream if stream is not None else _current_stream()
    o = opts if opts is not None else options()
    bound = g.rounds_bound()
    # first try: room for up to 65535 rounds but at most ~1 GB of counters
    # (many seeds); a run with more rounds reports it and is repeated
    cap = (min(bound, 65535, max(1024, (1 << 30) // (4 * max(s, 1))))
           if max_rounds is None else int(max_rounds))
    while True:
        counts = np.zeros((cap + 1, s), dtype=np.uint32)
        mact = np.zeros(cap + 2, dtype=np.uint64)
        c = _abi.Counts(s=s, max_rounds=cap, rounds=0, reserved=0,
                        counts=counts.ctypes.data, m_active=mact.ctypes.data)
        rc = fn(g._h, seeds.ctypes.data, s, ctypes.byref(c), ctypes.byref(o), st)
        if rc == _abi.PG_ERANGE and max_rounds is None and cap < bound:
            cap = bound
            continue
        _abi.check(rc, what)
        T = int(c.rounds)
        return Result(rounds=T, counts=counts[:T + 1].copy(), m_active=mact[:T + 2].copy(),
                      s=s, n=g.n)


def propagate_p(g: Graph, seeds, max_rounds: int | None = None, opts=None,
                stream=None) -> Result:
    """PROPAGATE-P (Alg. 1): all seeds diffuse together, s bits per node."""
    return _run(_abi.lib().pg_propagate_p, "pg_propagate_p", g, seeds, max_rounds, opts, stream)


def propagate_s(g: Graph, seeds, max_rounds: int | None = None, opts=None,
                stream=None) -> Result:
    """PROPAGATE-S (Alg. 2): seeds in passes of 1-bit planes, early break."""
    return _run(_abi.lib().pg_propagate_s, "pg_propagate_s", g, seeds, max_rounds, opts, stream)


def autotune(g: "Graph", seeds, max_trials: int = 24, opts=None, stream=None,
             algorithm: str = "p"):
    """pg_autotune: fastest schedule options for PROPAGATE-P (algorithm "p")
    or PROPAGATE-S ("s") on g with these seeds (counts checked identical
    across candidates). Returns (options, report dict)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    st = stream if stream is not None else _current_stream()
    o = opts if opts is not None else options()
    alg = {"p": _abi.PG_ALG_P, "s": _abi.PG_ALG_S}[algorithm]
    rep = _abi.TuneReport()
    _abi.check(_abi.lib().pg_autotune(g._h, seeds.ctypes.data, int(seeds.size), alg,
                                      int(max_trials), ctypes.byref(o), ctypes.byref(rep), st),
               "pg_autotune")
    return o, {f: getattr(rep, f) for f, _ in _abi.TuneReport._fields_}


class Batch:
    """pg_batch: PROPAGATE-P over many independent graphs, packed by
    signature width into disjoint unions that each run as one propagation.
    Host CSR arrays (over in-edges) and seeds are copied at add()."""

    def __init__(self):
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().pg_batch_create(ctypes.byref(h)), "pg_batch_create")
        self._h = h
        self._n = []
        self._s = []

    def add(self, row_ptr, col, seeds, n: int | None = None, directed: bool = True) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        sd = np.ascontiguousarray(seeds, dtype=np.int32)
        n = int(rp.size - 1 if n is None else n)
        idx = ctypes.c_int32(-1)
        _abi.check(_abi.lib().pg_batch_add(self._h, rp.ctypes.data, cl.ctypes.data, n,
                                           int(cl.size), int(bool(directed)), sd.ctypes.data,
                                           int(sd.size), ctypes.byref(idx)), "pg_batch_add")
        self._n.append(n)
        self._s.append(int(sd.size))
        return int(idx.value)

    def add_inputs(self, g, seeds) -> int:
        return self.add(g.row_ptr, g.col, seeds, n=g.n, directed=g.directed)

    def __len__(self):
        return len(self._n)

    def run(self, opts=None, stream=None):
        """Runs every graph; opts None = the tuned options (else defaults)."""
        st = stream if stream is not None else _current_stream()
        o = ctypes.byref(opts) if opts is not None else None
        _abi.check(_abi.lib().pg_batch_run(self._h, o, st), "pg_batch_run")

    def result(self, index: int) -> Result:
        """Counts and m_active of graph `index` from the last run (its own
        m_active, as if it had run alone)."""
        s, n = self._s[index], self._n[index]
        cap = min(max(n - 1, 0), 64)
        while True:
            counts = np.zeros((cap + 1, s), dtype=np.uint32)
            mact = np.zeros(cap + 2, dtype=np.uint64)
            c = _abi.Counts(s=s, max_rounds=cap, rounds=0, reserved=0,
                            counts=counts.ctypes.data, m_active=mact.ctypes.data)
            rc = _abi.lib().pg_batch_result(self._h, int(index), ctypes.byref(c))
            if rc == _abi.PG_ERANGE and c.rounds > cap:
                cap = int(c.rounds)  # the exact size, known now
                continue
            _abi.check(rc, "pg_batch_result")
            break
        T = int(c.rounds)
        return Result(rounds=T, counts=counts[:T + 1].copy(), m_active=mact[:T + 2].copy(),
                      s=s, n=n)

    def set_streams(self, streams: int):
        """pg_batch_set_streams: groups run at once (1 = one after another)."""
        _abi.check(_abi.lib().pg_batch_set_streams(self._h, int(streams)), "pg_batch_set_streams")

    def tune(self, max_trials: int = 24, stream=None) -> dict:
        """pg_batch_tune: picks schedule options per width class; later
        run() calls without opts use them."""
        st = stream if stream is not None else _current_stream()
        rep = _abi.TuneReport()
        _abi.check(_abi.lib().pg_batch_tune(self._h, int(max_trials), ctypes.byref(rep), st),
                   "pg_batch_tune")
        return {f: getattr(rep, f) for f, _ in _abi.TuneReport._fields_}

    def group_stats(self) -> list:
        """pg_stats dict per group of the last run (one per width class of
        packed graphs, one per graph run alone), narrowest first."""
        out, k = [], 0
        while True:
            st = _abi.Stats()
            if _abi.lib().pg_batch_group_stats(self._h, k, ctypes.byref(st)) != _abi.PG_OK:
                return out
            out.append({f: getattr(st, f) for f, _ in _abi.Stats._fields_})
            k += 1

    def group_options(self) -> list:
        """(graphs, options dict) per group, numbered as group_stats."""
        out, k = [], 0
        while True:
            o, ng = _abi.Options(), ctypes.c_int32(0)
            if _abi.lib().pg_batch_get_options(self._h, k, ctypes.byref(o),
                                               ctypes.byref(ng)) != _abi.PG_OK:
                return out
            out.append((int(ng.value), options_dict(o)))
            k += 1

    def stats(self) -> dict:
        st = _abi.BatchStats()
        _abi.check(_abi.lib().pg_batch_get_stats(self._h, ctypes.byref(st)), "pg_batch_get_stats")
        return {f: getattr(st, f) for f, _ in _abi.BatchStats._fields_}

    def close(self):
        if self._h:
            _abi.lib().pg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """pg_server: resident graphs and asynchronous PROPAGATE-P requests with
    continuous batching (merging of queued requests on one graph, and with
    cross_graph on graphs of one signature width as a packed union;
    concurrent slots; admission by device-memory budget). Results are the counts
    pg_propagate_p gives for each request alone."""

    def __init__(self, slots: int = 4, merge_max: int = 16, merge_max_seeds: int = 8192,
                 hbm_budget: int = 0, opts=None, cross_graph: bool = True):
        c = _abi.ServerConfig()
        _abi.lib().pg_server_default_config(ctypes.byref(c))
        c.slots, c.merge_max, c.merge_max_seeds, c.hbm_budget = (
            int(slots), int(merge_max), int(merge_max_seeds), int(hbm_budget))
        c.cross_graph = int(bool(cross_graph))
        if opts is not None:
            c.opt = opts
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().pg_server_create(ctypes.byref(c), ctypes.byref(h)),
                   "pg_server_create")
        self._h = h
        self._graph_n = {}
        self._req = {}  # request id -> (graph id, s)

    def add_graph(self, row_ptr, col, n: int | None = None, directed: bool = True) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        n = int(rp.size - 1 if n is None else n)
        gid = ctypes.c_int32(-1)
        _abi.check(_abi.lib().pg_server_add_graph(self._h, rp.ctypes.data, cl.ctypes.data, n,
                                                  int(cl.size), int(bool(directed)),
                                                  ctypes.byref(gid)), "pg_server_add_graph")
        self._graph_n[int(gid.value)] = n
        return int(gid.value)

    def add_inputs(self, g) -> int:
        return self.add_graph(g.row_ptr, g.col, n=g.n, directed=g.directed)

    def remove_graph(self, graph_id: int):
        _abi.check(_abi.lib().pg_server_remove_graph(self._h, int(graph_id)),
                   "pg_server_remove_graph")
        self._graph_n.pop(int(graph_id), None)

    def submit(self, graph_id: int, seeds) -> int:
        sd = np.ascontiguousarray(seeds, dtype=np.int32)
        rid = ctypes.c_int64(0)
        _abi.check(_abi.lib().pg_server_submit(self._h, int(graph_id), sd.ctypes.data,
                                               int(sd.size), ctypes.byref(rid)),
                   "pg_server_submit")
        self._req[int(rid.value)] = (int(graph_id), int(sd.size))
        return int(rid.value)

    @staticmethod
    def _info(i: _abi.RequestInfo) -> dict:
        return {f: getattr(i, f) for f, _ in _abi.RequestInfo._fields_}

    def poll(self, request_id: int) -> dict:
        info = _abi.RequestInfo()
        _abi.check(_abi.lib().pg_server_poll(self._h, int(request_id), ctypes.byref(info)),
                   "pg_server_poll")
        return self._info(info)

    def wait(self, request_id: int, timeout_ms: int = -1) -> dict | None:
        """Info once finished; None on timeout."""
        info = _abi.RequestInfo()
        rc = _abi.lib().pg_server_wait(self._h, int(request_id), int(timeout_ms),
                                       ctypes.byref(info))
        if rc == _abi.PG_ETIMEOUT:
            return None
        _abi.check(rc, "pg_server_wait")
        return self._info(info)

    def result(self, request_id: int, timeout_ms: int = -1):
        """Waits for the request and returns (Result, info); releases it."""
        info = self.wait(request_id, timeout_ms)
        if info is None:
            raise TimeoutError(f"request {request_id} not finished")
        gid, s = self._req[int(request_id)]
        n = self._graph_n[gid]
        cap = max(int(info["rounds"]), 0)  # T is known once the request is done
        counts = np.zeros((cap + 1, s), dtype=np.uint32)
        c = _abi.Counts(s=s, max_rounds=cap, rounds=0, reserved=0,
                        counts=counts.ctypes.data, m_active=None)
        out = _abi.RequestInfo()
        rc = _abi.lib().pg_server_result(self._h, int(request_id), ctypes.byref(c),
                                         ctypes.byref(out))
        if rc != _abi.PG_ERANGE:
            del self._req[int(request_id)]
        _abi.check(rc, "pg_server_result")
        T = int(c.rounds)
        res = Result(rounds=T, counts=counts[:T + 1].copy(),
                     m_active=np.zeros(T + 2, dtype=np.uint64), s=s, n=n)
        return res, self._info(out)

    def cancel(self, request_id: int):
        _abi.check(_abi.lib().pg_server_cancel(self._h, int(request_id)), "pg_server_cancel")

    def stats(self) -> dict:
        st = _abi.ServerStats()
        _abi.check(_abi.lib().pg_server_get_stats(self._h, ctypes.byref(st)),
                   "pg_server_get_stats")
        return {f: getattr(st, f) for f, _ in _abi.ServerStats._fields_}

    def close(self):
        if self._h:
            _abi.lib().pg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def progressive(g: "Graph", eps: float, rng_seed: int = 0, block: int = 256,
                stable_tol: float | None = None, opts=None, stream=None):
    """pg_progressive: PROPAGATE-P over seed blocks drawn uniformly without
    replacement until ceil(ln n / eps^2) seeds, or, with stable_tol, until the
    estimates settle (see include/propagate.h).

    Returns (Result over all drawn seeds, seeds, per-block metrics)."""
    n = g.n
    cols = max(1, min(n, int(np.ceil(np.log(max(n, 2)) / (eps * eps)))))
    st = stream if stream is not None else _current_stream()
    o = opts if opts is not None else options()
    cap = min(g.rounds_bound(), 65535, max(1024, (1 << 30) // (4 * cols)))
    seeds = np.zeros(cols, dtype=np.int32)
    counts = np.zeros((cap + 1, cols), dtype=np.uint32)
    mact = np.zeros(cap + 2, dtype=np.uint64)
    hist = (_abi.MetricsOut * (-(-cols // block)))()
    c = _abi.Counts(s=cols, max_rounds=cap, rounds=0, reserved=0, counts=counts.ctypes.data,
                    m_active=mact.ctypes.data)
    drawn, nblk = ctypes.c_int32(0), ctypes.c_int32(0)
    _abi.check(_abi.lib().pg_progressive(g._h, float(eps), int(block),
                                         float(stable_tol or 0.0), int(rng_seed),
                                         seeds.ctypes.data, ctypes.byref(drawn), ctypes.byref(c),
                                         hist, len(hist), ctypes.byref(nblk), ctypes.byref(o), st),
               "pg_progressive")
    k, T = int(drawn.value), int(c.rounds)
    res = Result(rounds=T, counts=np.ascontiguousarray(counts[:T + 1, :k]),
                 m_active=mact[:T + 2].copy(), s=k, n=n)
    history = []
    for b in range(int(nblk.value)):
        h = {f: getattr(hist[b], f) for f, _ in _abi.MetricsOut._fields_}
        h["seeds"] = min(k, (b + 1) * block) if b + 1 < nblk.value else k
        history.append(h)
    return res, seeds[:k].copy(), history


def metrics(res: Result, n: int | None = None, tau=(9, 10)) -> dict:
    """pg_metrics: diameter, effective diameter, average distance, reachable
    pairs and connectivity rate from a Result."""
    counts = np.ascontiguousarray(res.counts, dtype=np.uint32)
    c = _abi.Counts(s=res.s, max_rounds=res.rounds, rounds=res.rounds, reserved=0,
                    counts=counts.ctypes.data, m_active=None)
    out = _abi.MetricsOut()
    _abi.check(_abi.lib().pg_metrics(ctypes.byref(c), int(n if n is not None else res.n),
                                     int(tau[0]), int(tau[1]), ctypes.byref(out)), "pg_metrics")
    return {f: getattr(out, f) for f, _ in _abi.MetricsOut._fields_}
