"""Host-side pieces of bench.py: algorithmic bytes per kernel and the use of
the committed capture (void once a kernel's source changed)."""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _inp():
    n = 1000
    z = np.zeros(n, np.int64)
    li = [np.zeros(n, np.uint8), np.zeros(n, np.uint8)] + [z] * 4 + [np.zeros(n, np.int32)]
    return {"li": {"cols": li, "keys": [0, 1], "preds": [(6, 0, 1)]},
            "zipf": {"cols": [z, z], "keys": [0], "preds": []},
            "four": {"cols": [z, z], "keys": [0], "preds": []},
            "bk": z[:10], "bp": z[:10], "pk": z}


class _T:
    def __init__(self, n):
        self.n = n

    def numel(self):
        return self.n


def test_algorithmic_bytes():
    inp = _inp()
    res = {"zipf": (_T(7), [_T(7)] * 4), "join": (_T(900), _T(900), _T(900)),
           "zipf.records": 600}
    assert bench.algo_bytes("gb_stream", "zipf", inp, res) == 16_000
    assert bench.algo_bytes("gb_main_keyset", "zipf", inp, res) == 8_000
    assert bench.algo_bytes("gb_main_keyset", "lineitem", inp, res) == 1000 * (1 + 1 + 4)
    assert bench.algo_bytes("gb_part_hist", "zipf", inp, res) == 8_000
    assert bench.algo_bytes("gb_part_scatter", "zipf", inp, res) == 16_000 + 16 * 600
    assert bench.algo_bytes("gb_part_agg", "zipf", inp, res) == 16 * 600 + 7 * 8 * 5
    assert bench.algo_bytes("join_probe", "join", inp, res) == 8_000 + 900 * 16
    assert bench.algo_bytes("sketch", "zipf", inp, res) == 0


def test_capture_scaling_and_staleness(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source")
    (tmp_path / "profiles").mkdir()
    doc = {"kernels": {"gb_stream": {"source": str(src),
                                     "source_sha1": hashlib.sha1(b"kernel source").hexdigest(),
                                     "bytes_per_unit": 16.5, "warp_inst_per_unit": 2.0}}}
    (tmp_path / "profiles" / "kernel_traffic.txt").write_text(json.dumps(doc))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sz = bench.full_sizes(True)
    traffic, inst = bench.captured("gb_stream", "zipf", sz)
    assert traffic == 16.5 * sz["big"] and inst == 2.0 * sz["big"]
    assert bench.captured("gb_part_agg", "zipf", sz) == (None, None)
    src.write_text("kernel source, changed")
    assert bench.captured("gb_stream", "zipf", sz) == (None, None)


def test_capture_void_when_launch_host_code_changes(tmp_path, monkeypatch):
    kern, host = tmp_path / "k.cu", tmp_path / "api.cu"
    kern.write_text("kernel source")
    host.write_text("table sizing")
    (tmp_path / "profiles").mkdir()
    sha = lambda b: hashlib.sha1(b).hexdigest()
    doc = {"kernels": {"gb_main_keyset": {
        "sources": {str(kern): sha(b"kernel source"), str(host): sha(b"table sizing")},
        "bytes_per_unit": 10.0, "warp_inst_per_unit": 4.0}}}
    (tmp_path / "profiles" / "kernel_traffic.txt").write_text(json.dumps(doc))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sz = bench.full_sizes(True)
    assert bench.captured("gb_main_keyset", "zipf", sz) == (10.0 * sz["big"], 4.0 * sz["big"])
    host.write_text("table sizing, changed")
    assert bench.captured("gb_main_keyset", "zipf", sz) == (None, None)
    host.unlink()
    assert bench.captured("gb_main_keyset", "zipf", sz) == (None, None)


def test_cpu_legs_single_and_partitioned(monkeypatch):
    sz = dict(li=3000, nb=1000, np=6000, big=20_000)
    inp = bench.make_inputs(sz, seed=0)
    fr = {"lineitem": 1.0, "join": 0.5, "zipf": 0.5, "fourkeys": 0.5}
    one = bench.time_oracle_parts(inp, sz, fr)
    many = bench.time_oracle_parts(inp, sz, fr, threads=3)
    assert one.keys() == many.keys() == set(bench.PARTS)
    assert all(one[p][0] == many[p][0] and many[p][1] > 0 for p in one)
    rows_full = bench.part_rows(sz)
    line = bench.cpu_partitioned(inp, sz, rows_full, fr)
    assert line["value"] > 0 and line["cores"] >= 1 and line["unit"] == "rows/s"
    assert set(line["parts_rows_per_s"]) == set(bench.PARTS)

    from oracle import partitioned

    def boom(*a, **k):
        raise RuntimeError("planted")

    monkeypatch.setattr(partitioned, "groupby", boom)
    monkeypatch.setattr(partitioned, "default_threads", lambda: 2)
    assert bench.cpu_partitioned(inp, sz, rows_full, fr) == {"error": "RuntimeError: planted"}


def test_kernel_table_rates_and_shares():
    inp = _inp()
    res = {"zipf": (_T(7), [_T(7)] * 4), "join": (_T(900), _T(900), _T(900)),
           "zipf.records": 600}
    kern = {("zipf", "gb_main_keyset"): [2, 4.0], ("zipf", "sketch"): [1, 1.0],
            ("join", "join_probe"): [1, 0.5], ("zipf", "gb_part_scan"): [2, 0.0]}
    t = bench.kernel_table(kern, inp, res, peak_gbs=1.0)
    assert list(t) == ["zipf/gb_main_keyset", "zipf/sketch", "join/join_probe", "zipf/gb_part_scan"]
    assert abs(sum(d["share"] for d in t.values()) - 1.0) < 1e-12
    # 8000 B per launch in 2 ms
    assert abs(t["zipf/gb_main_keyset"]["algo_gbs"] - 8000 / 2e-3 / 1e9) < 1e-12
    assert t["zipf/gb_main_keyset"]["frac"] == t["zipf/gb_main_keyset"]["algo_gbs"]
    assert "algo_gbs" not in t["zipf/sketch"] and "algo_gbs" not in t["zipf/gb_part_scan"]
    assert abs(t["join/join_probe"]["algo_gbs"] - (8000 + 900 * 16) / 0.5e-3 / 1e9) < 1e-12
    # a kernel whose bytes cannot be derived keeps its timing only
    t = bench.kernel_table({("join", "gb_compact"): [1, 1.0]}, inp, {}, 1.0)
    assert t["join/gb_compact"] == {"launches": 1, "total_ms": 1.0, "share": 1.0}


def test_launch_units():
    sz = bench.full_sizes(False)
    assert bench.launch_units("zipf", sz) == 200_000_000
    assert bench.launch_units("join", sz) == 16_000_000
    assert bench.launch_units("lineitem", sz) == 1_000_000


def test_binding_roofline_picks_the_higher_utilisation():
    sz = bench.full_sizes(False)
    # 1.6 GB in 5 ms on a 6700 GB/s roof: 4.8 % of HBM; 2.35e9 warp instructions
    # in 5 ms against 152 x 4 x 2.07e9: 37 % of issue -> issue binds
    roof, instr = bench.binding_roofline("zipf", "gb_main_keyset", 1.6e9, 5.0, 6700.0, "measured",
                                         5.6e9, 2.35e9, 152, 2070.0, sz)
    assert roof["bound"] == "alu"
    assert abs(roof["frac"] - 2.35e9 / 5e-3 / (152 * 4 * 2.07e9)) < 1e-9
    assert abs(roof["hbm"]["frac"] - 1.6e9 / 5e-3 / 6700e9) < 1e-12
    assert abs(instr["warp_inst_per_row"] - 2.35e9 / 2e8) < 1e-9
    assert abs(instr["warp_inst_per_sector"] - 2.35e9 / (5.6e9 / 32)) < 1e-9
    # a streaming kernel: 3.2 GB in 0.6 ms (80 % of HBM), few instructions -> HBM binds
    roof, _ = bench.binding_roofline("fourkeys", "gb_stream", 3.2e9, 0.6, 6700.0, "measured",
                                     3.3e9, 4e8, 152, 2070.0, sz)
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["frac"] - 3.2e9 / 0.6e-3 / 6700e9) < 1e-12 and roof["issue_frac"] < roof["frac"]
    # no capture: HBM only
    roof, instr = bench.binding_roofline("zipf", "x", 1e9, 1.0, 6700.0, "measured", None, None,
                                         152, None, sz)
    assert roof["bound"] == "hbm" and instr is None
