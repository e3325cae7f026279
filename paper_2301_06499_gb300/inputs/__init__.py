"""Seeded synthetic inputs: CSR graphs over in-edges and seed samples.

This module holds none of the propagation method's arithmetic. It builds the
graphs and seed sets that both the CPU oracle (under ``oracle/``) and the CUDA
path consume, so that the two sides are fed identical inputs while sharing no
code.

Graph classes stand in for the paper's real datasets (Table 1): uniform sparse
(Erdos-Renyi), skewed web/social (R-MAT) and long-diameter lattices (grid).
Every random draw comes from one counter-based SplitMix64 stream (see
``gen.cpp``), so results are independent of the thread count and identical on
x86_64 and aarch64 hosts.

A CSR here is over in-edges: row ``v`` lists every ``u`` with an arc u -> v,
rows sorted ascending, no duplicates. Undirected graphs are stored symmetrised.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_SO = os.path.join(_HERE, "_pg_inputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.cpp into a host shared library next to it (g++, -O3)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Csr)
            lib.pgi_er.restype = P
            lib.pgi_er.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.pgi_rmat.restype = P
            lib.pgi_rmat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int]
            lib.pgi_grid.restype = P
            lib.pgi_grid.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_int]
            lib.pgi_csr_from_arcs.restype = P
            lib.pgi_csr_from_arcs.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int]
            lib.pgi_csr_free.restype = None
            lib.pgi_csr_free.argtypes = [P]
            lib.pgi_seeds.restype = ctypes.c_int
            lib.pgi_seeds.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_void_p]
            lib.pgi_rand.restype = ctypes.c_uint64
            lib.pgi_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


class _Owner:
    """Frees a C-allocated CSR once no numpy view of it is alive."""

    def __init__(self, lib, ptr):
        self._lib, self._ptr = lib, ptr

    def __del__(self):
        try:
            self._lib.pgi_csr_free(self._ptr)
        except Exception:
            pass


@dataclass
class Graph:
    """A CSR over in-edges. ``row_ptr`` int64[n+1], ``col`` int32[m]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    directed: bool
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def indegree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _wrap(ptr, directed: bool, name: str, **meta) -> Graph:
    if not ptr:
        raise MemoryError(f"input generator failed for {name}")
    lib = _load()
    c = ptr.contents
    n, m = int(c.n), int(c.m)
    owner = _Owner(lib, ptr)
    rp_buf = (ctypes.c_int64 * (n + 1)).from_address(ctypes.addressof(c.row_ptr.contents))
    col_buf = (ctypes.c_int32 * max(m, 1)).from_address(ctypes.addressof(c.col.contents))
    rp_buf._owner = owner
    col_buf._owner = owner
    row_ptr = np.frombuffer(rp_buf, dtype=np.int64, count=n + 1)
    col = np.frombuffer(col_buf, dtype=np.int32, count=m)
    return Graph(n=n, row_ptr=row_ptr, col=col, directed=directed, name=name, meta=meta)


def rand(seed: int, stream: int, index: int) -> int:
    """Value ``index`` of counter-based stream ``stream`` under ``seed``."""
    return int(_load().pgi_rand(seed, stream, index))


def er(n: int, avg_degree: float, seed: int, threads: int = 0) -> Graph:
    """Undirected G(n, M), M = round(n*avg_degree/2) pairs; loops dropped."""
    return _wrap(_load().pgi_er(n, avg_degree, seed, threads), False,
                 f"er_n{n}_d{avg_degree:g}_seed{seed}", kind="er", avg_degree=avg_degree,
                 seed=seed)


def rmat(scale: int, edge_factor: float, seed: int, directed: bool,
         a: float = 0.57, b: float = 0.19, c: float = 0.19, threads: int = 0) -> Graph:
    """R-MAT with 2**scale nodes and edge_factor * 2**scale edges (dedup)."""
    return _wrap(_load().pgi_rmat(scale, edge_factor, a, b, c, seed, int(directed), threads),
                 directed, f"rmat{'d' if directed else 'u'}_s{scale}_ef{edge_factor:g}_seed{seed}",
                 kind="rmat", scale=scale, edge_factor=edge_factor, seed=seed)


def grid(rows: int, cols: int, p_delete: float, seed: int, threads: int = 0) -> Graph:
    """rows x cols 4-neighbour lattice with each edge deleted w.p. p_delete."""
    return _wrap(_load().pgi_grid(rows, cols, p_delete, seed, threads), False,
                 f"grid_{rows}x{cols}_p{p_delete:g}_seed{seed}", kind="grid", rows=rows,
                 cols=cols, p_delete=p_delete, seed=seed)


def from_arcs(n: int, src, dst, symmetrise: bool = False, keep_self_loops: bool = True,
              name: str = "arcs") -> Graph:
    """CSR over in-edges of the arcs src[i] -> dst[i] (duplicates removed)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    ptr = _load().pgi_csr_from_arcs(n, src.size, src.ctypes.data, dst.ctypes.data,
                                    int(symmetrise), int(keep_self_loops), 0)
    return _wrap(ptr, not symmetrise, name, kind="arcs")


def seeds(n: int, s: int, seed: int) -> np.ndarray:
    """s distinct nodes of [0, n), uniform without replacement (Floyd)."""
    out = np.empty(s, dtype=np.int32)
    if _load().pgi_seeds(n, s, seed, out.ctypes.data) != 0:
        raise ValueError(f"cannot draw {s} distinct seeds from {n} nodes")
    return out


# ---------------------------------------------------------------- small graphs
def path(n: int, directed: bool = False) -> Graph:
    u = np.arange(n - 1, dtype=np.int32)
    return from_arcs(n, u, u + 1, symmetrise=not directed, name=f"path{n}")


def cycle(n: int) -> Graph:
    u = np.arange(n, dtype=np.int32)
    return from_arcs(n, u, (u + 1) % n, symmetrise=True, name=f"cycle{n}")


def star(n: int) -> Graph:
    leaves = np.arange(1, n, dtype=np.int32)
    return from_arcs(n, np.zeros(n - 1, np.int32), leaves, symmetrise=True, name=f"star{n}")


def complete(n: int) -> Graph:
    u, v = np.meshgrid(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32))
    keep = u != v
    return from_arcs(n, u[keep], v[keep], name=f"complete{n}")


def random_digraph(n: int, arcs: int, seed: int) -> Graph:
    """Directed multigraph sample: `arcs` uniform arcs (dedup, loops kept)."""
    src = np.array([rand(seed, 10, 2 * i) % n for i in range(arcs)], dtype=np.int32)
    dst = np.array([rand(seed, 10, 2 * i + 1) % n for i in range(arcs)], dtype=np.int32)
    return from_arcs(n, src, dst, name=f"digraph_n{n}_a{arcs}_seed{seed}")


# ------------------------------------------------------- sample-size policy
S_CLASSES = (64, 128, 256, 512)


def seeds_for_eps(n: int, eps: float) -> int:
    """Sample size ceil(ln n / eps^2), the Theta(ln n / eps^2) of Thm. 3 with
    constant 1."""
    return int(math.ceil(math.log(n) / (eps * eps)))


def s_class_for_eps(n: int, eps: float) -> int:
    """Smallest of {64,128,256,512} >= ceil(ln n/eps^2), capped at 512."""
    need = seeds_for_eps(n, eps)
    for s in S_CLASSES:
        if s >= need:
            return s
    return S_CLASSES[-1]


def s_rounded_64(n: int, eps: float) -> int:
    """ceil(ln n/eps^2) rounded up to a multiple of 64 (uncapped)."""
    need = seeds_for_eps(n, eps)
    return int(-(-need // 64) * 64)


@dataclass
class MixItem:
    graph: Graph
    s: int
    seeds: np.ndarray
    eps: float


def mix(count: int, n_lo: float, n_hi: float, seed: int, threads: int = 0) -> list:
    """Mixed batch of graphs: n log-uniform in [n_lo, n_hi]; type uniformly
    one of ER (average degree uniform in [4, 32]), R-MAT (edge factor uniform
    in [8, 16], 2**round(log2 n) nodes, directed or not with equal odds) or
    grid (side round(sqrt n), 5% deletion). Per graph eps is 0.1 or 0.2 and
    s = s_class_for_eps(n, eps); one graph in four instead takes s from
    {64, 128} so that every signature width occurs."""
    items = []
    for k in range(count):
        r = [rand(seed, 20, 8 * k + j) for j in range(8)]
        u01 = [(x >> 11) * (1.0 / (1 << 53)) for x in r]
        n = int(round(math.exp(math.log(n_lo) + u01[0] * (math.log(n_hi) - math.log(n_lo)))))
        kind = r[1] % 3
        gseed = seed * 1000003 + k
        if kind == 0:
            deg = 4.0 + 28.0 * u01[2]
            g = er(n, deg, gseed, threads)
        elif kind == 1:
            scale = max(4, int(round(math.log2(n))))
            ef = 8.0 + 8.0 * u01[2]
            g = rmat(scale, ef, gseed, directed=bool(r[3] & 1), threads=threads)
        else:
            side = max(2, int(round(math.sqrt(n))))
            g = grid(side, side, 0.05, gseed, threads)
        eps = 0.1 if (r[4] & 1) else 0.2
        if r[5] % 4 == 0:
            s = (64, 128)[r[6] & 1]
        else:
            s = s_class_for_eps(g.n, eps)
        s = min(s, g.n)
        items.append(MixItem(graph=g, s=s, seeds=seeds(g.n, s, gseed + 7), eps=eps))
    return items
