"""Summaries of Nsight Compute CSV output (``ncu --csv --log-file ...``).

  python ncu_summary.py launches <launches.csv>
      per kernel: launches, total device time, share (markdown table)
  python ncu_summary.py traffic <metrics.csv> [skip]
      per kernel: mean DRAM bytes (read + write) per launch, over its launches
      after the first `skip` of that kernel (JSON; `bench.py --write-traffic`
      turns such captures into profiles/pull_traffic.json)
"""
from __future__ import annotations

import collections
import csv
import json
import re
import sys

_UNIT_NS = {"nsecond": 1.0, "ns": 1.0, "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6,
            "second": 1e9, "s": 1e9}
_UNIT_B = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def _rows(path):
    with open(path) as f:
        lines = [ln for ln in f if not ln.startswith("==")]
    rows = list(csv.reader(lines))
    hdr = rows[0]
    idx = {h: i for i, h in enumerate(hdr)}
    for r in rows[1:]:
        if len(r) == len(hdr):
            yield {h: r[i] for h, i in idx.items()}


def short_name(kernel: str) -> str:
    """'void pg::k_pull<4, 4>(pg::Params)' -> 'k_pull<4, 4>'."""
    k = re.sub(r"^void\s+", "", kernel)
    k = k.split("(")[0]
    return k.split("::")[-1] if "<" not in k else re.sub(r"^.*::(?=[^:<]*<)", "", k)


def launches(path):
    tot = collections.OrderedDict()
    for r in _rows(path):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        ns = float(r["Metric Value"].replace(",", "")) * _UNIT_NS.get(r["Metric Unit"], 1.0)
        k = short_name(r["Kernel Name"])
        c = tot.setdefault(k, [0, 0.0])
        c[0] += 1
        c[1] += ns
    total = sum(v[1] for v in tot.values()) or 1.0
    return {k: {"launches": v[0], "total_ms": v[1] / 1e6, "share": v[1] / total}
            for k, v in sorted(tot.items(), key=lambda kv: -kv[1][1])}


def traffic_totals(path):
    """{kernel: (total DRAM bytes read + written, launches)} of one capture."""
    per = collections.defaultdict(lambda: collections.defaultdict(float))
    for r in _rows(path):
        m = r.get("Metric Name")
        if m not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        b = float(r["Metric Value"].replace(",", "")) * _UNIT_B.get(r["Metric Unit"], 1.0)
        per[short_name(r["Kernel Name"])][int(r["ID"])] += b
    return {k: (sum(v.values()), len(v)) for k, v in per.items()}


def traffic(path, skip: int = 0):
    per = collections.defaultdict(lambda: collections.defaultdict(float))
    for r in _rows(path):
        m = r.get("Metric Name")
        if m not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        b = float(r["Metric Value"].replace(",", "")) * _UNIT_B.get(r["Metric Unit"], 1.0)
        per[short_name(r["Kernel Name"])][int(r["ID"])] += b
    out = {}
    for k, v in per.items():
        ids = sorted(v)[skip:]
        if ids:
            out[k] = sum(v[i] for i in ids) / len(ids)
    return out


def main(argv):
    if len(argv) >= 2 and argv[0] == "launches":
        res = launches(argv[1])
        print("| kernel | launches | total ms (serialised, cold) | share |")
        print("|---|---:|---:|---:|")
        for k, v in res.items():
            print(f"| `{k}` | {v['launches']} | {v['total_ms']:.3f} | {v['share']:.3f} |")
        return 0
    if len(argv) >= 2 and argv[0] == "traffic":
        res = traffic(argv[1], int(argv[2]) if len(argv) > 2 else 0)
        print(json.dumps(res, indent=1))
        return 0
    print(__doc__)
    return 2


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
