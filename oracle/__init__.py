"""CPU oracle for PROPAGATE — test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package. The library's product path never does,
and this package imports nothing from the library: it shares no code with the
CUDA path. Inputs come from the seeded generators, which hold none of the
method's arithmetic.

Functions (all cite the passage they state; see ``oracle.c`` for the C):
  - ``seed_histograms``: per-seed BFS distance histograms, the exact per-round
    per-seed counts of PROPAGATE-P and -S (Sec. 4; rand-BFS of Sec. 5.1).
  - ``apsp_floyd_warshall``: all-pairs distances for tiny graphs.
  - ``m_active``: arcs read by the round-t sweep under the skip rule of the
    proof of Thm. 1, restated from distances.
  - ``metrics``: diameter, effective diameter, average distance, reachable
    pairs and connectivity rate (Sec. 3; last steps of Alg. 1).
  - ``propagate_p``: Alg. 1 itself on the host (s-bit signatures, sweep by
    sweep), a second statement of the per-seed counts and the paper's own
    method timed on the host cores.

The one pin that is NOT available is the paper's accuracy claim (Thm. 3,
Table 4): it needs the real datasets. Every function here is pinned by the
tests against closed forms, Floyd-Warshall and hand-computed examples.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a host shared library (gcc -O2)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", _SRC,
                    "-o", tmp], check=True)
    os.replace(tmp, _SO)
    return _SO


class MetricsOut(ctypes.Structure):
    _fields_ = [("diameter", ctypes.c_int32), ("eff_diameter", ctypes.c_int32),
                ("eff_diameter_interp", ctypes.c_double), ("avg_distance", ctypes.c_double),
                ("avg_distance_incl_self", ctypes.c_double),
                ("connectivity_rate", ctypes.c_double), ("reachable_pairs", ctypes.c_double),
                ("R_last", ctypes.c_uint64), ("dist_sum", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.or_seed_histograms.restype = ctypes.c_int
            lib.or_seed_histograms.argtypes = [i64, vp, vp, vp, i64, i64, vp, vp, vp,
                                               ctypes.c_int]
            lib.or_apsp_floyd_warshall.restype = ctypes.c_int
            lib.or_apsp_floyd_warshall.argtypes = [i64, vp, vp, vp]
            lib.or_m_active.restype = ctypes.c_int
            lib.or_m_active.argtypes = [i64, vp, vp, vp, i64, i64, vp, ctypes.c_int]
            lib.or_propagate_p.restype = ctypes.c_int
            lib.or_propagate_p.argtypes = [i64, vp, vp, vp, i64, i64, vp, vp, vp, ctypes.c_int]
            lib.or_metrics.restype = ctypes.c_int
            lib.or_metrics.argtypes = [vp, i64, i64, i64, i64, i64,
                                       ctypes.POINTER(MetricsOut)]
            _lib = lib
    return _lib


def _threads(threads):
    return threads if threads and threads > 0 else (os.cpu_count() or 1)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    return int(g.n), rp, col


def _check(rc, what):
    if rc == -1:
        raise ValueError(f"oracle {what}: invalid arguments")
    if rc == -2:
        raise MemoryError(f"oracle {what}: out of memory")
    if rc == -3:
        raise OverflowError(f"oracle {what}: a distance exceeds the histogram capacity")
    if rc != 0:
        raise RuntimeError(f"oracle {what}: status {rc}")


def seed_histograms(g, seeds, cap: int | None = None, threads: int = 0,
                    with_distances: bool = False):
    """Per-seed BFS distance histograms.

    Returns ``hist`` int64[s, T+1] with hist[i, d] = |{v : d(x_i, v) = d}| and
    T the largest finite distance from any seed (the diameter lower bound of
    Alg. 1), plus ``ecc`` int32[s]. With ``with_distances`` also the node-major
    distance matrix int32[n, s] (-1 = unreachable)."""
    n, rp, col = _csr(g)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    s = seeds.size
    cap = int(cap if cap is not None else n)
    cap = max(1, min(cap, n))
    hist = np.zeros((s, cap), dtype=np.int64)
    ecc = np.zeros(s, dtype=np.int32)
    dmat = np.empty((n, s), dtype=np.int32) if with_distances else None
    rc = _load().or_seed_histograms(n, rp.ctypes.data, col.ctypes.data, seeds.ctypes.data, s,
                                    cap, hist.ctypes.data, ecc.ctypes.data,
                                    dmat.ctypes.data if dmat is not None else None,
                                    _threads(threads))
    _check(rc, "seed_histograms")
    T = int(ecc.max()) if s else 0
    hist = np.ascontiguousarray(hist[:, :T + 1])
    if with_distances:
        return hist, ecc, dmat
    return hist, ecc


def apsp_floyd_warshall(g) -> np.ndarray:
    """All-pairs distances (n x n, -1 unreachable); tiny graphs only."""
    n, rp, col = _csr(g)
    dist = np.empty((n, n), dtype=np.int64)
    _check(_load().or_apsp_floyd_warshall(n, rp.ctypes.data, col.ctypes.data, dist.ctypes.data),
           "apsp_floyd_warshall")
    return dist


def m_active(g, dmat: np.ndarray, rounds: int, threads: int = 0) -> np.ndarray:
    """uint64[rounds+1]: arcs read by the round-t sweep (entry 0 is 0)."""
    n, rp, col = _csr(g)
    dmat = np.ascontiguousarray(dmat, dtype=np.int32)
    s = dmat.shape[1]
    out = np.zeros(rounds + 1, dtype=np.uint64)
    _check(_load().or_m_active(n, rp.ctypes.data, col.ctypes.data, dmat.ctypes.data, s, rounds,
                               out.ctypes.data, _threads(threads)), "m_active")
    return out


def propagate_p(g, seeds, cap: int | None = None, threads: int = 0,
                with_m_active: bool = False):
    """Alg. 1 on the host: returns (counts uint32[T+1, s], T), counts[t, i] =
    the nodes seed i's bit reached in round t (its nodes at distance t), and
    with ``with_m_active`` also m_active uint64[T+2] as the sweeps find it."""
    n, rp, col = _csr(g)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    s = seeds.size
    cap = int(cap if cap is not None else n)
    counts = np.zeros((cap + 1, s), dtype=np.uint32)
    mact = np.zeros(cap + 2, dtype=np.uint64)
    T = ctypes.c_int32(0)
    _check(_load().or_propagate_p(n, rp.ctypes.data, col.ctypes.data, seeds.ctypes.data, s, cap,
                                  counts.ctypes.data, ctypes.byref(T), mact.ctypes.data,
                                  _threads(threads)),
           "propagate_p")
    out = (np.ascontiguousarray(counts[:T.value + 1]), int(T.value))
    if with_m_active:
        return out + (np.ascontiguousarray(mact[:T.value + 2]),)
    return out


def metrics(hist: np.ndarray, n: int, tau_num: int = 9, tau_den: int = 10) -> dict:
    """Metrics of Sec. 3 / Alg. 1 from per-seed histograms int64[s, cap]."""
    hist = np.ascontiguousarray(hist, dtype=np.int64)
    s, cap = hist.shape
    out = MetricsOut()
    _check(_load().or_metrics(hist.ctypes.data, s, cap, n, tau_num, tau_den, ctypes.byref(out)),
           "metrics")
    return {f: getattr(out, f) for f, _ in MetricsOut._fields_}


def run(g, seeds, threads: int = 0, tau=(9, 10), with_m_active: bool = True,
        with_distances: bool = False) -> dict:
    """Everything the GPU path returns, for one graph and seed set:
    counts (uint32[T+1, s], row t = per-seed new nodes at hop t), rounds T,
    m_active (uint64[T+2], the final empty sweep included) and metrics; with
    ``with_distances`` also "dmat", the node-major distances int32[n, s]."""
    if with_m_active or with_distances:
        hist, ecc, dmat = seed_histograms(g, seeds, threads=threads, with_distances=True)
    else:
        hist, ecc = seed_histograms(g, seeds, threads=threads)
    T = hist.shape[1] - 1
    res = {
        "rounds": T,
        "counts": np.ascontiguousarray(hist.T.astype(np.uint32)),
        "metrics": metrics(hist, g.n, *tau),
    }
    if with_m_active:
        res["m_active"] = m_active(g, dmat, T + 1, threads=threads)
    if with_distances:
        res["dmat"] = dmat
    return res
