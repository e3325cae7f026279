"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares; host-only entry points work on CPU. No compute call here
touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2301_06499_gb300 as pg
from paper_2301_06499_gb300 import _abi
from paper_2301_06499_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = _abi.lib()
    names = _declared("propagate.h")
    assert "pg_propagate_p" in names and "pg_propagate_s" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(_abi.SIGNATURES)


def test_version_strerror_options():
    lib = _abi.lib()
    assert b"sm_103a" in lib.pg_version()
    assert lib.pg_strerror(-7) == b"more rounds than max_rounds"
    o = pg.options()
    assert o.direction == pg.PG_DIR_AUTO and o.group_lanes == 0
    assert o.planes_per_pass == 64 and o.use_graphs == 1
    with pytest.raises(TypeError):
        pg.options(bogus=1)


def _metrics_from_hist(hist, n, tau=(9, 10)):
    counts = np.ascontiguousarray(hist.T.astype(np.uint32))
    res = pg.Result(rounds=hist.shape[1] - 1, counts=counts,
                    m_active=np.zeros(hist.shape[1] + 1, np.uint64), s=hist.shape[0], n=n)
    return pg.metrics(res, n, tau)


@pytest.mark.parametrize("seed", range(5))
def test_pg_metrics_matches_oracle(seed):
    g = I.er(400 + 50 * seed, 2.0 + seed, seed) if seed % 2 else I.random_digraph(300, 700, seed)
    s = 10 + 7 * seed
    seeds = I.seeds(g.n, s, seed + 40)
    hist, _ = oracle.seed_histograms(g, seeds)
    want = oracle.metrics(hist, g.n)
    got = _metrics_from_hist(hist, g.n)
    for k in ("diameter", "eff_diameter", "R_last", "dist_sum"):
        assert got[k] == want[k], k
    for k in ("eff_diameter_interp", "avg_distance", "avg_distance_incl_self",
              "connectivity_rate", "reachable_pairs"):
        assert got[k] == pytest.approx(want[k], rel=1e-12, abs=0.0), k


def test_pg_metrics_rejects_bad_input():
    lib = _abi.lib()
    counts = np.ones((1, 2), np.uint32)
    c = _abi.Counts(s=2, max_rounds=0, rounds=0, reserved=0, counts=counts.ctypes.data,
                    m_active=None)
    out = _abi.MetricsOut()
    assert lib.pg_metrics(ctypes.byref(c), 10, 11, 10, ctypes.byref(out)) == _abi.PG_EINVAL
    assert lib.pg_metrics(ctypes.byref(c), 0, 9, 10, ctypes.byref(out)) == _abi.PG_EINVAL
    c.rounds = 3  # more rows than the buffer claims
    assert lib.pg_metrics(ctypes.byref(c), 10, 9, 10, ctypes.byref(out)) == _abi.PG_EINVAL


def test_pg_metrics_p4_worked_example():
    g = I.path(4)
    hist, _ = oracle.seed_histograms(g, np.arange(4, dtype=np.int32))
    m = _metrics_from_hist(hist, 4)
    assert m["eff_diameter"] == 3 and m["diameter"] == 3
    assert m["eff_diameter_interp"] == pytest.approx(2.2, rel=1e-14)
    assert m["reachable_pairs"] == 16.0


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror in _abi.py has the C header's size and field
    offsets (compiled with the host C compiler against include/propagate.h),
    so no field of the boundary is read at the wrong place."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = {"pg_options": _abi.Options, "pg_counts": _abi.Counts,
             "pg_metrics_out": _abi.MetricsOut, "pg_stats": _abi.Stats,
             "pg_tune_report": _abi.TuneReport, "pg_batch_stats": _abi.BatchStats,
             "pg_server_config": _abi.ServerConfig, "pg_request_info": _abi.RequestInfo,
             "pg_server_stats": _abi.ServerStats, "pg_generator": _abi.Generator}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "propagate.h"',
             "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, cls in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_argument_checks_before_any_device_work():
    """Bad arguments are refused with PG_EINVAL before the device is touched,
    and without a GPU a valid graph is refused with PG_ECUDA: the library has
    no host fallback for the propagation."""
    L = _abi.lib()
    out = ctypes.c_void_p()
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    assert L.pg_graph_from_csr(None, None, 10, 0, 1, 0, None, ctypes.byref(out)) == _abi.PG_EINVAL
    assert L.pg_graph_from_csr(rp.ctypes.data, col.ctypes.data, 0, 2, 1, 0, None,
                               ctypes.byref(out)) == _abi.PG_EINVAL
    assert L.pg_graph_from_csr(rp.ctypes.data, col.ctypes.data, 2, -1, 1, 0, None,
                               ctypes.byref(out)) == _abi.PG_EINVAL
    # past the largest graph whose rounds one 64-bit counter holds (changed
    # rows in 27 bits, their out-arcs in 37): refused before the arrays are read
    for n, m in ((1 << 27, 2), (2, 1 << 37)):
        assert L.pg_graph_from_csr(rp.ctypes.data, col.ctypes.data, n, m, 1, 0, None,
                                   ctypes.byref(out)) == _abi.PG_EINVAL
    gen = _abi.Generator(kind=1, directed=0, seed=1, scale=27, edge_factor=1.0,
                         a=0.57, b=0.19, c=0.19)
    assert L.pg_graph_generate(ctypes.byref(gen), 0, None, ctypes.byref(out)) == _abi.PG_EINVAL
    c = _abi.Counts(s=1, max_rounds=0, rounds=0, reserved=0, counts=None, m_active=None)
    assert L.pg_propagate_p(None, None, 1, ctypes.byref(c), None, None) == _abi.PG_EINVAL
    assert L.pg_propagate_s(None, None, 1, ctypes.byref(c), None, None) == _abi.PG_EINVAL
    assert L.pg_batch_create(None) == _abi.PG_EINVAL
    bh = ctypes.c_void_p()
    assert L.pg_batch_create(ctypes.byref(bh)) == _abi.PG_OK
    for bad in (0, -1, 17):
        assert L.pg_batch_set_streams(bh, bad) == _abi.PG_EINVAL
    assert L.pg_batch_set_streams(bh, 1) == _abi.PG_OK
    assert L.pg_batch_set_streams(None, 4) == _abi.PG_EINVAL
    sd = np.array([0], np.int32)
    assert L.pg_batch_add(bh, rp.ctypes.data, col.ctypes.data, 1 << 27, 2, 1, sd.ctypes.data, 1,
                          None) == _abi.PG_EINVAL
    L.pg_batch_free(bh)
    assert L.pg_server_create(None, None) == _abi.PG_EINVAL
    assert L.pg_autotune(None, None, 1, 0, 1, None, None, None) == _abi.PG_EINVAL
    import torch
    if not torch.cuda.is_available():
        rc = L.pg_graph_from_csr(rp.ctypes.data, col.ctypes.data, 2, 2, 1, 0, None,
                                 ctypes.byref(out))
        assert rc == _abi.PG_ECUDA


def test_debug_bounds_variant_builds_and_exports_every_symbol():
    """The PG_DEBUG_BOUNDS build (every gather checks its indices and records
    a bad one instead of faulting) compiles for sm_103a and exports the same
    C ABI."""
    import ctypes as C
    from paper_2301_06499_gb300 import build
    path = build.build(variant="debug-bounds")
    assert path != build.lib_path("") and path.endswith("libpropagate_debug_bounds.so")
    lib = C.CDLL(path)
    for name in _declared("propagate.h"):
        assert hasattr(lib, name), name
