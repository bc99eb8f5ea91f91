"""Summaries of ncu captures of this library's kernels (a development tool;
it reads captures taken on a GB300 with `ncu ... -o FILE`).

    python -m paper_2608_13696_gb300.ncu_summary [--traffic FILE] \\
        CAPTURE.ncu-rep=ID:UNITS:UNIT[:ALGO_BYTES] ...
    python -m paper_2608_13696_gb300.ncu_summary --launches LAUNCHES.csv

ID is the kernel's name in bench.py's kernel table (e.g. gb_part_scatter),
UNITS how many rows (or probes, groups, ...) the captured launch processed,
ALGO_BYTES its algorithmic bytes (inputs read once, outputs written once).
For every capture this prints one markdown table row: time, DRAM bytes and
GB/s, algorithmic GB/s, warp instructions issued per unit and per
algorithmic byte, issue-slot and warp occupancy, L2 and L1 hit rates and the
three largest stall reasons per issued instruction.  With --traffic it
writes, per ID, the DRAM bytes and issued warp instructions per unit and
the SHA-1 of the sources that build and size the kernel (bench.py uses a
record only while those sources are unchanged).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = "paper_2608_13696_gb300/csrc/"

# kernel id -> the sources that compile it and size its launch
SOURCES = {
    "gb_main_keyset": ["distinct.cu", "api.cu"],
    "gb_part_hist": ["stream.cu", "api.cu"],
    "gb_part_scatter": ["stream.cu", "api.cu"],
    "gb_part_l2": ["stream.cu", "api.cu"],
    "gb_part_scan": ["groupby.cu", "api.cu"],
    "gb_part_agg": ["groupby.cu", "api.cu"],
    "gb_compact": ["groupby.cu", "api.cu"],
    "gb_main_regs": ["groupby.cu", "api.cu"],
    "gb_main_layered": ["groupby.cu", "api.cu"],
    "gb_main_staged_keyset": ["groupby.cu", "api.cu"],
    "gb_stream": ["stream.cu", "api.cu"],
    "join_build": ["join.cu", "api.cu"],
    "join_probe": ["join.cu", "api.cu"],
    "sketch": ["sketch.cu", "api.cu"],
    "mlp_forward": ["mlp.cu", "api.cu"],
    "mlp_backward_sample": ["mlp.cu", "api.cu"],
    "mlp_backward": ["mlp.cu", "api.cu"],
    "mlp_adamw": ["mlp.cu", "api.cu"],
    "batch_a": ["batch.cu", "batch_api.cu"],
    "batch_b": ["batch.cu", "batch_api.cu"],
    "shard_scatter": ["shard.cu"],
    "hll": ["distinct.cu", "api.cu"],
}

METRICS = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "smsp__inst_issued.sum", "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "sm__warps_active.avg.pct_of_peak_sustained_active", "lts__t_sector_hit_rate.pct",
    "l1tex__t_sector_hit_rate.pct", "sm__cycles_elapsed.avg.per_second",
    "launch__registers_per_thread", "launch__grid_size", "launch__block_size",
    "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_lg_throttle_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_membar_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_branch_resolving_per_issue_active.ratio",
]
# ncu --metrics argument for a capture that this tool can summarise
METRICS_ARG = ",".join(METRICS)

_SCALE = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-9,
          "usecond": 1e-6, "msecond": 1e-3, "second": 1, "ns": 1e-9, "us": 1e-6, "ms": 1e-3,
          "s": 1, "hz": 1, "Khz": 1e3, "Mhz": 1e6, "Ghz": 1e9}


def read_capture(path: str) -> dict:
    """The first launch's metrics of an ncu capture, in base units (bytes,
    seconds, hertz)."""
    out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True,
                         text=True, check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr, units, first = rows[0], rows[1], rows[2]
    m = {"kernel": first[hdr.index("Kernel Name")]}
    for name in METRICS:
        if name not in hdr:
            continue
        i = hdr.index(name)
        v = first[i].replace(",", "")
        try:
            m[name] = float(v) * _SCALE.get(units[i], 1)
        except ValueError:
            pass
    return m


def summarize(m: dict, units: float, algo_bytes: float | None) -> dict:
    t = m["gpu__time_duration.sum"]
    dram = m.get("dram__bytes_read.sum", 0) + m.get("dram__bytes_write.sum", 0)
    inst = m.get("smsp__inst_issued.sum")
    stalls = {k.split("stalled_")[1].split("_per_issue")[0]: v for k, v in m.items()
              if "issue_stalled" in k}
    top = sorted(stalls.items(), key=lambda kv: -kv[1])[:3]
    return {"kernel": m["kernel"], "us": t * 1e6, "dram_bytes": dram, "dram_gbs": dram / t / 1e9,
            "algo_gbs": algo_bytes / t / 1e9 if algo_bytes else None,
            "warp_inst": inst, "inst_per_unit": inst / units if inst else None,
            "inst_per_byte": inst / algo_bytes if inst and algo_bytes else None,
            "issue_pct": m.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
            "warps_pct": m.get("sm__warps_active.avg.pct_of_peak_sustained_active"),
            "l2_hit_pct": m.get("lts__t_sector_hit_rate.pct"),
            "l1_hit_pct": m.get("l1tex__t_sector_hit_rate.pct"),
            "regs": m.get("launch__registers_per_thread"), "stalls": top}


def _f(x, fmt):
    return "-" if x is None else format(x, fmt)


def table_row(kid: str, s: dict, units: float, unit: str) -> str:
    stalls = ", ".join(f"{k} {v:.1f}" for k, v in s["stalls"])
    return (f"| `{kid}` | {s['kernel'][:48]} | {units:.3g} {unit} | {s['us']:.1f} | "
            f"{s['dram_bytes'] / 1e6:.0f} | {s['dram_gbs']:.0f} | {_f(s['algo_gbs'], '.0f')} | "
            f"{_f(s['inst_per_unit'], '.2f')} | {_f(s['inst_per_byte'], '.3f')} | "
            f"{_f(s['issue_pct'], '.0f')} % | {_f(s['warps_pct'], '.0f')} % | "
            f"{_f(s['l2_hit_pct'], '.0f')} % | {_f(s['l1_hit_pct'], '.0f')} % | "
            f"{_f(s['regs'], '.0f')} | {stalls} |")


HEADER = ("| id | kernel | units | us | DRAM MB | DRAM GB/s | algorithmic GB/s | warp inst / unit"
          " | warp inst / algo byte | issue active | warps active | L2 hit | L1 hit | regs"
          " | top stalls (per issue) |\n" + "|---" * 15 + "|")


def sha1(rel_path: str) -> str:
    return hashlib.sha1(open(os.path.join(ROOT, rel_path), "rb").read()).hexdigest()


def launch_table(csv_path: str, skip_prefixes=("at::", "void at::")) -> str:
    """Markdown table of an `ncu --metrics gpu__time_duration.sum --csv
    --log-file` launch list: per kernel, launches, total time, share of the
    library's kernel time, grid x block (torch's own kernels left out)."""
    rows = [r for r in csv.reader(open(csv_path)) if len(r) > 10]
    hdr = rows[0]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    gi, bi = hdr.index("Grid Size"), hdr.index("Block Size")
    agg = {}
    for r in rows[1:]:
        name = r[ki]
        if name.startswith(skip_prefixes):
            continue
        t = float(r[vi].replace(",", "")) * _SCALE.get(r[ui], 1e-9)
        short = name.replace("(anonymous namespace)::", "").replace("unnamed>::", "")
        short = short.replace("void ", "").replace("rel::", "").split("(")[0]
        a = agg.setdefault(short, [0, 0.0, r[gi] + " x " + r[bi]])
        a[0] += 1
        a[1] += t
    total = sum(v[1] for v in agg.values()) or 1.0
    lines = ["| kernel | launches | total us | share | grid x block |", "|---|---|---|---|---|"]
    for k, (n, t, gb) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        lines.append(f"| `{k}` | {n} | {t * 1e6:.1f} | {100 * t / total:.1f} % | {gb} |")
    lines.append(f"\nTotal {total * 1e6:.1f} us over {sum(v[0] for v in agg.values())} library launches.")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2608_13696_gb300.ncu_summary")
    ap.add_argument("captures", nargs="*", help="FILE.ncu-rep=ID:UNITS:UNIT[:ALGO_BYTES]")
    ap.add_argument("--traffic", default=None, help="JSON record for bench.py")
    ap.add_argument("--launches", default=None, help="launch-list CSV to tabulate")
    a = ap.parse_args(argv)
    if a.launches:
        print(launch_table(a.launches))
        if not a.captures:
            return 0
    record = {"note": "DRAM bytes (read + write) and issued warp instructions per unit from one "
                      "ncu capture per kernel (paper_2608_13696_gb300.profile_cases); bench.py "
                      "scales them by its own launch's units and drops a record once one of "
                      "its sources changed", "kernels": {}}
    print(HEADER)
    for spec in a.captures:
        path, rest = spec.split("=", 1)
        parts = rest.split(":")
        kid, units, unit = parts[0], float(parts[1]), parts[2]
        algo = float(parts[3]) if len(parts) > 3 else None
        s = summarize(read_capture(path), units, algo)
        print(table_row(kid, s, units, unit))
        srcs = {CSRC + f: sha1(CSRC + f) for f in SOURCES.get(kid, [])}
        record["kernels"][kid] = {
            "capture_kernel": s["kernel"], "sources": srcs, "unit": unit, "units": units,
            "dram_bytes": s["dram_bytes"], "bytes_per_unit": s["dram_bytes"] / units,
            "warp_inst": s["warp_inst"], "warp_inst_per_unit": s["inst_per_unit"]}
    if a.traffic:
        with open(a.traffic, "w") as f:
            json.dump(record, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
