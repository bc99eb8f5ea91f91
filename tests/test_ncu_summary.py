"""Host logic of the ncu summary tool (no profiler, no GPU): per-capture
arithmetic and the launch-list table."""
import csv

import pytest

from paper_2608_13696_gb300 import ncu_summary as N


def test_summarize_rates_and_stalls():
    m = {"kernel": "k", "gpu__time_duration.sum": 2e-3, "dram__bytes_read.sum": 3e9,
         "dram__bytes_write.sum": 1e9, "smsp__inst_issued.sum": 8e8,
         "smsp__issue_active.avg.pct_of_peak_sustained_active": 40.0,
         "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio": 5.0,
         "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio": 1.0,
         "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio": 3.0,
         "smsp__average_warps_issue_stalled_membar_per_issue_active.ratio": 0.5}
    s = N.summarize(m, units=1e8, algo_bytes=2e9)
    assert s["us"] == pytest.approx(2000.0)
    assert s["dram_bytes"] == 4e9
    assert s["dram_gbs"] == pytest.approx(2000.0)   # 4 GB in 2 ms
    assert s["algo_gbs"] == pytest.approx(1000.0)
    assert s["inst_per_unit"] == pytest.approx(8.0)
    assert s["inst_per_byte"] == pytest.approx(0.4)
    assert [k for k, _ in s["stalls"]] == ["long_scoreboard", "barrier", "wait"]
    row = N.table_row("id", s, 1e8, "rows")
    assert row.startswith("| `id` | k | 1e+08 rows | 2000.0 | 4000 | 2000 | 1000 | 8.00 | 0.400 | 40 % |")


def test_summarize_without_algorithmic_bytes():
    m = {"kernel": "k", "gpu__time_duration.sum": 1e-6, "dram__bytes_read.sum": 0.0}
    s = N.summarize(m, units=1, algo_bytes=None)
    assert s["algo_gbs"] is None and s["inst_per_unit"] is None
    assert "| - |" in N.table_row("id", s, 1, "x")


def test_launch_table_sums_per_kernel_and_drops_torch(tmp_path):
    path = tmp_path / "launches.csv"
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name",
           "Metric Unit", "Metric Value"]
    rows = [
        ["0", "1", "p", "h", "void rel::(anonymous namespace)::a_k<long>(P)", "1", "7", "(256, 1, 1)",
         "(304, 1, 1)", "0", "10.3", "s", "gpu__time_duration.sum", "usecond", "3"],
        ["1", "1", "p", "h", "void rel::(anonymous namespace)::a_k<long>(P)", "1", "7", "(256, 1, 1)",
         "(304, 1, 1)", "0", "10.3", "s", "gpu__time_duration.sum", "usecond", "2"],
        ["2", "1", "p", "h", "b_k(P)", "1", "7", "(128, 1, 1)", "(2, 1, 1)", "0", "10.3", "s",
         "gpu__time_duration.sum", "nsecond", "4,000"],
        ["3", "1", "p", "h", "void at::native::elementwise_kernel<128>(int)", "1", "7",
         "(128, 1, 1)", "(1, 1, 1)", "0", "10.3", "s", "gpu__time_duration.sum", "usecond", "50"],
    ]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(hdr)
        w.writerows(rows)
    t = N.launch_table(str(path))
    lines = t.splitlines()
    assert lines[2] == "| `a_k<long>` | 2 | 5.0 | 55.6 % | (304, 1, 1) x (256, 1, 1) |"
    assert lines[3] == "| `b_k` | 1 | 4.0 | 44.4 % | (2, 1, 1) x (128, 1, 1) |"
    assert "elementwise" not in t
    assert "Total 9.0 us over 3 library launches." in t
