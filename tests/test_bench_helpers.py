"""Host-side helpers of bench.py (no GPU): the pull kernel names it matches
against ncu's launch lists, the per-kernel source hashes that key the stored
DRAM-traffic figures, and the table written from ncu CSV captures."""
import json

import bench


def _st(**kw):
    st = {"words_per_row": 4, "words_per_gather": 4, "group_lanes": 16, "pass_words": 1}
    st.update(kw)
    return st


def test_kernel_names_follow_the_instantiations():
    assert bench.kernel_name(_st()) == "k_pull<4, 16, 0>"
    assert bench.kernel_name(_st(pass_words=4)) == "k_pull<4, 16, 1>"
    assert bench.kernel_name(_st(words_per_gather=1, group_lanes=8)) == "k_pull<1, 8, 0>"
    for wp, nw in ((16, 1), (64, 2), (88, 3), (128, 4), (1568, 0)):
        st = _st(words_per_row=wp, words_per_gather=0)
        assert bench.kernel_name(st) == f"k_pull_wide<{nw}, 0>"
        assert bench.kernel_name(dict(st, pass_words=87)) == f"k_pull_wide<{nw}, 1>"
    # statistics of a batch carry no pass_words: plain PROPAGATE-P kernels
    st = _st()
    del st["pass_words"]
    assert bench.kernel_name(st) == "k_pull<4, 16, 0>"


def test_kernel_hash_covers_each_kernels_own_sources():
    h4 = bench.kernel_hash("k_pull<4, 16, 1>")
    assert h4 == bench.kernel_hash("k_pull<4, 4, 0>")  # one source file per words class
    assert h4 != bench.kernel_hash("k_pull<8, 16, 0>")
    assert bench.kernel_hash("k_pull_wide<0, 1>") == bench.kernel_hash("k_pull_wide<3, 0>")
    assert bench.kernel_hash("k_pull_wide<0, 1>") not in (h4, bench.kernel_hash("k_pull<1, 8, 0>"))


def test_write_traffic_from_ncu_csv(tmp_path):
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = []
    for i, (k, rd, wr) in enumerate((("void pg::k_pull<4, 16, 1>(pg::Params)", "300", "100"),
                                     ("void pg::k_pull<4, 16, 1>(pg::Params)", "500", "100"),
                                     ("void k_post<1, 0>(Params)", "50", "50"))):
        rows.append(f'"{i}","{k}","dram__bytes_read.sum","Mbyte","{rd}"\n')
        rows.append(f'"{i}","{k}","dram__bytes_write.sum","Mbyte","{wr}"\n')
    csv = tmp_path / "t.csv"
    csv.write_text("==PROF== Connected\n" + hdr + "".join(rows))
    out_path = tmp_path / "traffic.json"
    out = bench.write_traffic("rmat22_directed_s256", [str(csv)], str(out_path))
    stored = json.loads(out_path.read_text())
    assert stored == out
    assert stored["bytes_per_launch"]["k_pull<4, 16, 1>"] == 500e6  # mean of 400 and 600 MB
    assert stored["kernel_hash"]["k_pull<4, 16, 1>"] == bench.kernel_hash("k_pull<4, 16, 1>")


def test_round_bytes_follow_the_per_round_formula():
    """|A|(8 + 2 s/8) + m_active (4 + s/8) + |F| 4 for PROPAGATE-P; per pass of
    64 planes (8-byte signatures) for PROPAGATE-S."""
    st = {"active_rows": 10, "m_active_total": 100, "changed_rows": 7}
    assert bench.round_bytes(st, 512, False) == 10 * (8 + 128) + 100 * (4 + 64) + 7 * 4
    assert bench.round_bytes(st, 512, True) == 10 * (8 + 16) + 100 * (4 + 8) + 7 * 4
    assert bench.round_bytes(st, 32, True) == 10 * (8 + 8) + 100 * (4 + 4) + 7 * 4


def test_load_traffic_keeps_only_figures_of_the_current_sources(tmp_path):
    """A stored DRAM figure counts as this build's traffic only while the
    kernel's sources hash as they did at the capture; otherwise it is kept
    apart as an earlier build's, with both hashes."""
    cur = bench.kernel_hash("k_pull<8, 16, 0>")
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps({
        "workload": "w",
        "kernel_hash": {"k_pull<8, 16, 0>": cur, "k_pull<8, 16, 1>": "0123456789ab"},
        "bytes_per_launch": {"k_pull<8, 16, 0>": 4.0e10, "k_pull<8, 16, 1>": 4.2e10}}))
    table, earlier = bench.load_traffic("w", str(path))
    assert table == {"k_pull<8, 16, 0>": 4.0e10}
    assert earlier == {"k_pull<8, 16, 1>": {"bytes_per_launch": 4.2e10,
                                            "sources_hash": "0123456789ab",
                                            "current_sources_hash":
                                                bench.kernel_hash("k_pull<8, 16, 1>")}}
    assert bench.load_traffic("other", str(path)) == ({}, {})
    assert bench.load_traffic("w", str(tmp_path / "missing.json")) == ({}, {})
    # the committed table: each figure lands on exactly one side
    t2, e2 = bench.load_traffic("rmat26_undirected_s512")
    assert set(t2) | set(e2) and not set(t2) & set(e2)
