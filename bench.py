#!/usr/bin/env python3
"""Throughput of the relational hot path on one GB300 (or N replicas).

One step = one pass over every built operator on seeded synthetic columns
(they stand in for the TPC-H data the paper profiles, Sec. 3.2):
  lineitem  fused filter (date <= 2430) + group-by (flag, status), 5 exact
            int64 aggregates, 10^6 rows (plan: exact distinct count)
  join      hash build of 10^6 unique int64 keys + probe of 1.6*10^7 keys
            (90 % present) emitting (probe_idx, build_idx, payload)
  zipf      group-by of 2*10^8 (int64 key, int64 value) rows, keys
            Zipf(1.1) over 10^7 ranks, sum/count/min/max (plan: exact count)
  fourkeys  the same with 4 distinct keys
Every call goes through the C ABI of librel.so.  value = rows of all parts /
device time of the step (inputs resident in HBM); e2e = the same through the
public API with the inputs copied from pinned host memory and the results
copied back inside the timed region.  The step reads 6.6 GB, far more than
the 129 MB L2, so consecutive steps do not hit a warm cache.

--impl reference times the CPU oracle (single-threaded C++) on bounded row
prefixes of the same parts and extrapolates each part's rows/s linearly.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rows/s & %HBM/instr-issue roofline, groupby+join probe; learned/batched vs plain"
WORKLOAD = ("lineitem filter+group-by 1e6 rows; join build 1e6 x probe 1.6e7; "
            "group-by 2e8 rows Zipf(1.1) over 1e7 keys; group-by 2e8 rows 4 keys")


def full_sizes(small: bool):
    if small:
        return dict(li=100_000, nb=100_000, np=1_600_000, big=20_000_000)
    return dict(li=1_000_000, nb=1_000_000, np=16_000_000, big=200_000_000)


# ----------------------------------------------------------------- inputs

def make_inputs(sz, seed, prefix=None):
    """Seeded inputs; with prefix = {part: fraction} only those leading rows
    (identical to the full columns' prefixes: the generator is counter-based)."""
    import synth
    from paper_2608_13696_gb300.workloads import kv_query, lineitem_query

    f = prefix or {}
    n = lambda key, part: max(1, int(sz[key] * f.get(part, 1.0)))
    li = synth.lineitem(n("li", "lineitem"), seed=seed)
    bk, bp = synth.join_build(sz["nb"], seed=seed)
    pk, _ = synth.join_probe(n("np", "join"), sz["nb"], seed=seed)
    zk, zv = synth.zipf_kv(n("big", "zipf"), seed=seed)
    fk, fv = synth.few_keys_kv(n("big", "fourkeys"), n_keys=4, seed=seed)
    return {"li": lineitem_query(li), "bk": bk, "bp": bp, "pk": pk,
            "zipf": kv_query(zk, zv), "four": kv_query(fk, fv)}


def part_rows(sz):
    return {"lineitem": sz["li"], "join": sz["nb"] + sz["np"], "zipf": sz["big"],
            "fourkeys": sz["big"]}


def part_bytes(inp):
    b = {"lineitem": sum(c.nbytes for c in inp["li"]["cols"]),
         "join": inp["bk"].nbytes + inp["bp"].nbytes + inp["pk"].nbytes,
         "zipf": sum(c.nbytes for c in inp["zipf"]["cols"]),
         "fourkeys": sum(c.nbytes for c in inp["four"]["cols"])}
    return b


# ------------------------------------------------------------- GPU parts

class GpuStep:
    """Device-resident inputs and the calls of one step."""

    def __init__(self, inp, dev):
        import torch

        from paper_2608_13696_gb300 import rel

        self.torch, self.rel, self.dev = torch, rel, dev
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        self.q = {}
        for name, key in (("lineitem", "li"), ("zipf", "zipf"), ("fourkeys", "four")):
            q = dict(inp[key])
            q["cols"] = [t(c) for c in inp[key]["cols"]]
            self.q[name] = q
        self.bk, self.bp, self.pk = t(inp["bk"]), t(inp["bp"]), t(inp["pk"])
        self.host = inp
        self.results = {}
        self.learned = False
        self.ws = {}

    def tensors(self):
        out = [self.bk, self.bp, self.pk]
        for q in self.q.values():
            out += q["cols"]
        return out

    def part(self, name):
        rel = self.rel
        if name == "join":
            tab = rel.JoinTable(self.bk, self.bp)
            self.results[name] = tab.probe(self.pk, capacity=self.pk.numel())
            return
        q = self.q[name]
        if self.learned:
            # learned sizing (sketch + planner network) in one call, with the
            # exact re-plan inside the call when the estimate overflows
            if name not in self.ws:
                self.ws[name] = rel._ws(rel.auto_ws_bytes(q), self.dev)
            keys, aggs, plan = rel.groupby_auto(q, flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH,
                                                ws=self.ws[name])
            self.results[name] = (keys, aggs)
            self.results[name + ".plan"] = plan
            return
        plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
        self.results[name] = rel.groupby(q, plan=plan)
        self.results[name + ".plan"] = plan

    def count_records(self):
        """Rows a partitioned plan writes as records (not pinned, not
        INT64_MIN) -- the partition passes' algorithmic traffic."""
        torch = self.torch
        for name in ("zipf", "fourkeys"):
            plan = self.results.get(name + ".plan")
            if plan is None or plan.variant != self.rel.VAR_PARTITIONED:
                continue
            k = self.q[name]["cols"][0]
            hot = torch.tensor([plan.hot_keys[i] for i in range(plan.n_hot)] +
                               [-(1 << 63)], dtype=torch.int64, device=k.device)
            self.results[name + ".records"] = int(k.numel() - torch.isin(k, hot).sum().item())

    def result_tensors(self):
        out = []
        for name in ("lineitem", "zipf", "fourkeys"):
            k, aggs = self.results[name]
            out += [k, *aggs]
        out += list(self.results["join"])
        return out


PARTS = ("lineitem", "join", "zipf", "fourkeys")
# bytes the kernel must move per unit, by (part, kernel): inputs read once,
# outputs written once; hash-table traffic is not algorithmic
def algo_bytes(kernel, part, inp, res):
    cols = {"lineitem": inp["li"]["cols"], "zipf": inp["zipf"]["cols"],
            "fourkeys": inp["four"]["cols"]}
    if (kernel.startswith("gb_main_") and kernel != "gb_main_keyset") or kernel == "gb_stream":
        return sum(c.nbytes for c in cols[part])
    if kernel == "gb_main_keyset":
        q = {"lineitem": inp["li"], "zipf": inp["zipf"], "fourkeys": inp["four"]}[part]
        used = set(q["keys"]) | {p[0] for p in q.get("preds", [])}
        return sum(q["cols"][c].nbytes for c in used)
    if kernel == "gb_compact":
        k, aggs = res[part]
        return (k.numel() * 8) * (1 + len(aggs))
    if kernel == "join_build":
        return inp["bk"].nbytes + inp["bp"].nbytes
    if kernel == "join_probe":
        return inp["pk"].nbytes + res["join"][0].numel() * 16
    # partitioned variant: histogram reads the keys; scatter reads key and
    # value and writes a 16-byte record per row that is not pinned;
    # aggregation reads the records and writes the groups
    if part in cols:
        recs = res.get(part + ".records", cols[part][0].shape[0])
        if kernel == "gb_part_hist":
            return cols[part][0].nbytes
        if kernel == "gb_part_scatter":
            return sum(c.nbytes for c in cols[part]) + 16 * recs
        if kernel == "gb_part_l2":  # level-1 records read, final records written
            return 32 * recs
        if kernel == "gb_part_agg":
            k, aggs = res[part]
            return 16 * recs + k.numel() * 8 * (1 + len(aggs))
    return 0


def captured(kernel, part, sz):
    """(DRAM bytes, warp instructions) per launch of `kernel` from the
    committed ncu capture (profiles/kernel_traffic.txt: per row or probe of a
    5e7-row case, scaled by this launch's rows); (None, None) when the
    kernel's source or its launch's host code changed since the capture, or
    there is none."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "kernel_traffic.txt")
    if not os.path.exists(path):
        return None, None
    k = json.load(open(path))["kernels"].get(kernel)
    if not k:
        return None, None
    # the kernel's source and the host code that sizes its launch (tables,
    # grid) must be the ones the counters were taken from
    srcs = k.get("sources") or {k["source"]: k["source_sha1"]}
    for rel_path, digest in srcs.items():
        src = os.path.join(ROOT, rel_path)
        if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != digest:
            return None, None
    units = launch_units(part, sz)
    return k["bytes_per_unit"] * units, k.get("warp_inst_per_unit", 0.0) * units or None


def launch_units(part, sz):
    """Rows (probe rows for the join) one launch of the part's hot kernel covers."""
    return {"lineitem": sz["li"], "join": sz["np"], "zipf": sz["big"], "fourkeys": sz["big"]}[part]


NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def kernel_table(kern, inp, res, peak_gbs):
    """Per (part, kernel): launches, total ms, share of kernel time and, where
    the kernel has algorithmic bytes, their rate and its fraction of peak_gbs."""
    total = sum(v[1] for v in kern.values()) or 1.0
    out = {}
    for (p, k), (n, ms) in sorted(kern.items(), key=lambda kv: -kv[1][1]):
        d = {"launches": n, "total_ms": ms, "share": ms / total}
        try:
            b = algo_bytes(k, p, inp, res)
        except (KeyError, IndexError, TypeError):
            b = 0
        if b and n and ms > 0:
            d["algo_gbs"] = b / (ms / n / 1e3) / 1e9
            d["frac"] = d["algo_gbs"] / peak_gbs
        out[f"{p}/{k}"] = d
    return out


def binding_roofline(part, kernel, abytes, ms_per_launch, peak_gbs, peak_src, traffic, winst,
                     n_sm, sm_mhz, sz):
    """The dominant kernel on both roofs of the paper's model (Sec. 2.2): HBM
    (algorithmic bytes / time / measured copy bandwidth) and instruction issue
    (warp instructions / time / (N_SM x 4 schedulers x SM clock sampled during
    the run)).  The binding roof is the one with the higher utilisation; the
    other is kept beside it.  Warp instructions and DRAM traffic come from the
    committed ncu capture (None when it no longer matches the source)."""
    from paper_2608_13696_gb300 import roofline as rf

    units = launch_units(part, sz)
    clock = sm_mhz * 1e6 if sm_mhz else None
    rep = rf.report(seconds=ms_per_launch / 1e3, algo_bytes=abytes,
                    peak_bytes_per_s=peak_gbs * 1e9, warp_inst=winst, n_sm=n_sm,
                    clock_hz=clock, dram_bytes=traffic, rows=units)
    hbm = {"achieved": rep["gbps"], "peak": peak_gbs, "unit": "GB/s", "frac": rep["hbm_frac"],
           "peak_source": peak_src, "frac_nominal": rep["gbps"] / NOMINAL_HBM_GBS,
           "peak_nominal": NOMINAL_HBM_GBS}
    instr = None
    if "issue_frac" in rep:
        issue_peak = rf.inst_throughput(n_sm, 4, clock)
        instr = {"kernel": f"{part}/{kernel}", "achieved_warp_inst_per_s": winst / (ms_per_launch / 1e3),
                 "peak_warp_inst_per_s": issue_peak, "frac": rep["issue_frac"],
                 "warp_inst_per_sector": rep.get("inst_per_sector"),
                 "warp_inst_per_row": rep.get("warp_inst_per_row"),
                 "warp_inst_per_byte": rep.get("inst_per_byte"),
                 "ridge_inst_per_sector": rf.ridge(issue_peak, peak_gbs * 1e9),
                 "n_sm": n_sm, "sm_mhz": sm_mhz, "source": "profiles/kernel_traffic.txt"}
    roof = {"kernel": f"{part}/{kernel}", "algo_bytes_per_launch": abytes,
            "ms_per_launch": ms_per_launch, "traffic": traffic}
    if instr and instr["frac"] > hbm["frac"]:
        # instruction issue binds: "alu" against N_SM x 4 x clock warp inst/s
        roof.update(bound="alu", achieved=instr["achieved_warp_inst_per_s"] / 1e9,
                    peak=instr["peak_warp_inst_per_s"] / 1e9, unit="G warp-inst/s",
                    frac=instr["frac"], hbm=hbm)
    else:
        roof.update(bound="hbm", achieved=hbm["achieved"], peak=peak_gbs, unit="GB/s",
                    frac=hbm["frac"], peak_source=peak_src, frac_nominal=hbm["frac_nominal"],
                    peak_nominal=NOMINAL_HBM_GBS)
        if instr:
            roof["issue_frac"] = instr["frac"]
    return roof, instr


# ----------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU (oracle)

def time_oracle_parts(inp, sz, frac_rows, threads: int = 1):
    """Time the oracle on row prefixes; returns {part: (rows, seconds)}.
    threads > 1: the oracle on hash partitions of the rows, one thread each
    (oracle.partitioned; results left in partition order)."""
    import oracle

    if threads > 1:
        from oracle import partitioned

        groupby = lambda q: partitioned.groupby(q, threads=threads, sort=False)
        join = lambda b, y, p: partitioned.join(b, y, p, threads=threads, sort=False)
    else:
        groupby, join = oracle.groupby, oracle.join
    out = {}
    n = max(1, int(sz["li"] * frac_rows["lineitem"]))
    q = dict(inp["li"])
    q["cols"] = [c[:n] for c in q["cols"]]
    t = time.perf_counter()
    groupby(q)
    out["lineitem"] = (n, time.perf_counter() - t)
    npr = max(1, int(sz["np"] * frac_rows["join"]))
    t = time.perf_counter()
    join(inp["bk"], inp["bp"], inp["pk"][:npr])
    out["join"] = (sz["nb"] + npr, time.perf_counter() - t)
    for name, key in (("zipf", "zipf"), ("fourkeys", "four")):
        n = max(1, int(sz["big"] * frac_rows[name]))
        q = dict(inp[key])
        q["cols"] = [c[:n] for c in q["cols"]]
        t = time.perf_counter()
        groupby(q)
        out[name] = (n, time.perf_counter() - t)
    return out


def cpu_partitioned(inp, sz, rows_full, fracs):
    """The multi-core CPU figure: the oracle per hash partition on every host
    core, on the same row prefixes as the single-core baseline.  A failure is
    reported in the line, not raised (it is context, not the measurement)."""
    try:
        from oracle import partitioned

        threads = partitioned.default_threads()
        t = time_oracle_parts(inp, sz, fracs, threads=threads)
        v, _ = extrapolate(t, rows_full)
        parts = {p: r / s for p, (r, s) in t.items()}
        return {"value": v, "unit": "rows/s", "cores": threads,
                "kind": "oracle per hash partition, one thread each",
                "sample": sample_text(fracs, sz), "parts_rows_per_s": parts}
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def extrapolate(timings, rows_full):
    """rows/s of a full step from per-part rates."""
    secs = sum(rows_full[p] / (r / s) for p, (r, s) in timings.items())
    return sum(rows_full.values()) / secs, secs


CPU_FRACS = {"lineitem": 1.0, "join": 0.5, "zipf": 0.25, "fourkeys": 0.25}
REF_FRACS = {"lineitem": 0.2, "join": 0.0625, "zipf": 0.01, "fourkeys": 0.01}


def sample_text(fr, sz):
    return (f"oracle on row prefixes: lineitem {int(sz['li'] * fr['lineitem'])}, join build "
            f"{sz['nb']} + probe {int(sz['np'] * fr['join'])}, zipf "
            f"{int(sz['big'] * fr['zipf'])}, fourkeys {int(sz['big'] * fr['fourkeys'])} rows; "
            f"each part's rows/s extrapolated linearly to the full step")


# ------------------------------------------------------------------- main

def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (every rank calls this; world 1: unchanged)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(rows_per_step: int, world: int, steps: int, ms: float) -> float:
    """Rows of all ranks' steps per second of the slowest rank (replicas:
    every rank runs its own full step, weak scaling)."""
    return rows_per_step * world * steps / (ms / 1e3)


def run_reference(args, sz):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    inp = make_inputs(sz, seed=0, prefix=REF_FRACS)
    rows_full = part_rows(sz)
    for _ in range(args.warmup):
        time_oracle_parts(inp, sz, REF_FRACS)
    t0 = time.perf_counter()
    tot = {p: [0, 0.0] for p in PARTS}
    for _ in range(args.steps):
        for p, (r, s) in time_oracle_parts(inp, sz, REF_FRACS).items():
            tot[p][0] += r
            tot[p][1] += s
    wall = time.perf_counter() - t0
    value, secs = extrapolate({p: tuple(v) for p, v in tot.items()}, rows_full)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(rows_full.values()) / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generators standing in for TPC-H)",
            "config": {"workload": WORKLOAD, "rows_per_step": sum(rows_full.values())},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle",
                             "sample": sample_text(REF_FRACS, sz)},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--small", action="store_true", help="10x smaller workload (quick checks)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--learned", type=int, default=2000,
                    help="instances of the learned-sizing comparison (0 = skip)")
    ap.add_argument("--no-learned-step", action="store_true",
                    help="skip the step timed with learned plans")
    ap.add_argument("--no-scale", action="store_true",
                    help="skip the 1e8-row lineitem run and the host-link measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-plain comparison")
    args = ap.parse_args()
    sz = full_sizes(args.small)
    if args.impl == "reference":
        return run_reference(args, sz)

    import torch
    import torch.distributed as dist

    from paper_2608_13696_gb300 import rel

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rel.load()

    inp = make_inputs(sz, seed=rank)
    rows_full = part_rows(sz)
    rows_step = sum(rows_full.values())
    g = GpuStep(inp, dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step(timing=None):
        for p in PARTS:
            c0 = rel.launch_count()
            if timing is not None:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
            g.part(p)
            if timing is not None:
                ev1 = torch.cuda.Event(enable_timing=True)
                ev1.record(stream)
                timing.append((p, ev0, ev1, rel.launch_count() - c0))

    for _ in range(args.warmup):
        step()
    barrier()

    timing = []
    with Clocks(local) as clk:
        rel.profile_start()
        l0 = rel.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step(timing)
        e1.record(stream)
        barrier()
        launches = rel.launch_count() - l0
        recs = rel.profile_stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_step = ms / args.steps
    value = whole_job_rate(rows_step, world, args.steps, ms)

    # per part and per kernel
    parts, kern = {}, {}
    i = 0
    for p, a, b, n in timing:
        d = parts.setdefault(p, {"ms": 0.0, "launches": 0})
        d["ms"] += a.elapsed_time(b) / args.steps
        d["launches"] += n
        for name, kms in recs[i:i + n]:
            kk = kern.setdefault((p, name), [0, 0.0])
            kk[0] += 1
            kk[1] += kms
        i += n
    for p, d in parts.items():
        d["rows"] = rows_full[p]
        d["rows_per_s"] = rows_full[p] / (d["ms"] / 1e3)
        d["launches"] //= args.steps
    (dp, dk), (dn, dms) = max(kern.items(), key=lambda kv: kv[1][1])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak_gbs = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    per_launch_ms = dms / dn
    g.count_records()
    abytes = algo_bytes(dk, dp, inp, g.results)
    traffic, winst = captured(dk, dp, sz)
    kernels = kernel_table(kern, inp, g.results, peak_gbs)
    clocks = clk.summary()

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof, instr = binding_roofline(dp, dk, abytes, per_launch_ms, peak_gbs, peak_src, traffic,
                                   winst, sms, clocks.get("sm_mhz"), sz)
    line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generators standing in for TPC-H)",
            "config": {"workload": WORKLOAD, "rows_per_step": rows_step,
                       "l2": "inputs larger than L2 (6.6 GB read per step)",
                       "plans": "exact distinct-count pre-pass (the plain form) + 4096-row sample sketch"},
            "parts": parts, "roofline": roof,
            "gpu_launches": launches, "kernels": kernels, "clocks": clocks}
    if instr:
        line["instr_roofline"] = instr

    if not args.no_e2e:
        line["e2e"] = run_e2e(args, g, inp, stream, world, barrier, rows_step)
    if rank == 0 and not args.no_learned_step:
        line["learned_step"] = run_learned_step(args, g, stream, rows_step, ms_step)
    if rank == 0 and not args.no_scale:
        line["lineitem_1e8"] = run_lineitem_scale(args, dev, peak_gbs)
        line["h2d_link"] = measure_h2d(dev)
    if rank == 0 and not args.no_cpu_baseline:
        t = time_oracle_parts(inp, sz, CPU_FRACS)
        v, _ = extrapolate(t, rows_full)
        line["cpu_baseline"] = {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                                "sample": sample_text(CPU_FRACS, sz),
                                "parts_rows_per_s": {p: r / s for p, (r, s) in t.items()},
                                "sample_s": sum(s for _, s in t.values())}
        line["cpu_partitioned"] = cpu_partitioned(inp, sz, rows_full, CPU_FRACS)
    if rank == 0 and args.learned > 0:
        line["learned"] = run_learned(args)
    if rank == 0 and not args.no_batched:
        line["batched"] = run_batched(args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_learned_step(args, g, stream, rows_step, plain_ms_step):
    """The same step with every group-by planned by the learned form (sketch +
    planner network; an overflowing estimate is re-planned exactly inside the
    call), device-timed like the plain step, results compared part by part
    with the plain step's."""
    import torch

    from paper_2608_13696_gb300 import planner, rel

    if not os.path.exists(planner.DEFAULT_WEIGHTS):
        return {"skipped": "no trained planner network"}
    planner.use_default()
    plain = {p: g.results[p] for p in ("lineitem", "zipf", "fourkeys")}
    g.learned = True
    try:
        for _ in range(max(1, args.warmup)):
            for p in PARTS:
                g.part(p)
        torch.cuda.synchronize()
        parts = {p: 0.0 for p in PARTS}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for p in PARTS:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.part(p)
                b.record(stream)
                b.synchronize()
                parts[p] += a.elapsed_time(b) / args.steps
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        mismatches, fell_back = 0, []
        for p, (k0, a0) in plain.items():
            k1, a1 = g.results[p]
            s0, o0 = torch.sort(k0)
            s1, o1 = torch.sort(k1)
            same = torch.equal(s0, s1) and all(torch.equal(x[o0], y[o1]) for x, y in zip(a0, a1))
            mismatches += not same
            if g.results[p + ".plan"].flags & rel.PLAN_FELL_BACK:
                fell_back.append(p)
    finally:
        g.learned = False
    return {"value": rows_step / (ms / 1e3), "unit": "rows/s", "ms_per_step": ms,
            "plain_ms_per_step": plain_ms_step, "speedup_vs_plain": plain_ms_step / ms,
            "parts_ms": parts, "mismatches": mismatches, "fell_back": fell_back,
            "plans": "learned sizing (sketch + network, exact re-plan on overflow) + sketch pins"}


def run_lineitem_scale(args, dev, peak_gbs):
    """The lineitem filter + group-by at 1e8 rows (3.8 GB, far above L2): the
    fused kernel's stable roofline figure, device-timed over 5 launches."""
    import torch

    import synth
    from paper_2608_13696_gb300 import rel
    from paper_2608_13696_gb300.workloads import lineitem_query

    n = 100_000_000 if not args.small else 10_000_000
    li = synth.lineitem(n, seed=7)
    q = lineitem_query(li)
    q["cols"] = [torch.from_numpy(c).to(dev) for c in q["cols"]]
    nbytes = sum(c.numel() * c.element_size() for c in q["cols"])
    del li
    plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    for _ in range(3):
        rel.groupby(q, plan=plan)
    torch.cuda.synchronize()
    rel.profile_start()
    for _ in range(5):
        rel.groupby(q, plan=plan)
    torch.cuda.synchronize()
    recs = rel.profile_stop()
    kern = {}
    for name, ms in recs:
        kern.setdefault(name, []).append(ms)
    main_k = max(kern, key=lambda k: sum(kern[k]))
    ms = float(np.mean(kern[main_k]))
    gbs = nbytes / (ms / 1e3) / 1e9
    out = {"rows": n, "bytes": nbytes, "kernel": main_k, "ms_per_launch": ms, "algo_gbs": gbs,
           "frac": gbs / peak_gbs, "frac_nominal": gbs / NOMINAL_HBM_GBS,
           "rows_per_s": n / (ms / 1e3), "groups": int(plan.est_groups),
           "plan": "exact distinct count + sketch pins (thread-private shared words)"}
    del q
    torch.cuda.empty_cache()
    return out


def measure_h2d(dev):
    """Pinned host -> device copy rate alone (1 GiB, best of 5), against which
    the end-to-end figure's copies can be read."""
    import torch

    h = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    best = None
    for _ in range(5):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        d.copy_(h, non_blocking=True)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    del h, d
    return {"bytes": 1 << 30, "ms": best, "gbs": (1 << 30) / (best / 1e3) / 1e9,
            "how": "one cudaMemcpyAsync of 1 GiB from pinned host memory, best of 5"}


def run_learned(args):
    """Learned sizing (sketch + planner network) against the plain exact
    pre-pass, on instances of 1e6..5e7 rows (uniform, Zipf 0.5/1/1.5,
    clustered keys) the network was not trained on; results compared."""
    from paper_2608_13696_gb300 import planner

    if not os.path.exists(planner.DEFAULT_WEIGHTS):
        return {"skipped": "no trained planner network"}
    n = args.learned if not args.small else min(args.learned, 20)
    r = planner.evaluate(range(1_000_000, 1_000_000 + n), with_labels=False, log_every=0,
                         rows_hi=50_000_000 if not args.small else 5_000_000, with_rows=False)
    r.pop("per_instance", None)
    r["timing"] = "wall clock per instance (plan + run + result count), inputs resident, L2 flushed"
    r["workload"] = (f"{n} unseen planner-workload instances (rows log-U[1e6, 5e7], uniform / "
                     f"Zipf 0.5, 1.0, 1.5 / clustered keys, domains log-U[10, 1e8])")
    return r


def run_batched(args):
    """The batched workload (4096 group-bys + 512 join partitions) as one
    graph-replayed batch against one call sequence per instance."""
    import torch

    from paper_2608_13696_gb300 import batched, planner, rel
    from synth import gpu as G

    if not os.path.exists(planner.DEFAULT_WEIGHTS):
        return {"skipped": "no trained planner network"}
    planner.use_default()
    recipe = G.batch_recipe(0) if not args.small else G.batch_recipe(0, 512, 64)
    gb, jn = G.batch_inputs(recipe)
    torch.cuda.synchronize()
    r = batched.measure(gb, jn, reps=3, autotune=True,
                        candidates=[c for c in rel.BATCH_SEARCH if c[2] in (1, 2)])
    r["config"] = list(r["config"])
    r["workload"] = (f"{len(gb)} group-bys (rows log-U[1e3,4e6], groups log-U[1,1e5], int32/int64 "
                     f"keys, sum+count) + {len(jn)} join partitions (build log-U[1e3,2.56e5], "
                     f"probe log-U[8e3,2e6], 90% hits)")
    del gb, jn
    torch.cuda.empty_cache()
    return r


def run_e2e(args, g, inp, stream, world, barrier, rows_step):
    """Same step through the public API with inputs from pinned host memory
    and every result copied back, copies inside the timed region.  The
    copies are pipelined with the work: each part's inputs go up on a copy
    stream in part order and the part starts when its own inputs have
    arrived; each part's results go down on another stream while the next
    part runs."""
    import torch

    part_in = {"lineitem": g.q["lineitem"]["cols"], "join": [g.bk, g.bp, g.pk],
               "zipf": g.q["zipf"]["cols"], "fourkeys": g.q["fourkeys"]["cols"]}
    host_in = {p: [t.cpu().pin_memory() for t in ts] for p, ts in part_in.items()}
    h2d = sum(t.numel() * t.element_size() for ts in host_in.values() for t in ts)
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    host_out = {}  # pinned result buffers, reused across steps
    d2h = [0]

    def pinned_like(key, o):
        b = host_out.get(key)
        if b is None or b.numel() < o.numel() or b.dtype != o.dtype:
            b = torch.empty(max(1, o.numel()), dtype=o.dtype, pin_memory=True)
            host_out[key] = b
        return b[:o.numel()]

    def results_of(p):
        if p == "join":
            return list(g.results["join"])
        k, aggs = g.results[p]
        return [k, *aggs]

    def e2e_step():
        arrived = {}
        with torch.cuda.stream(up):
            for p in PARTS:
                for h, d in zip(host_in[p], part_in[p]):
                    d.copy_(h, non_blocking=True)
                arrived[p] = torch.cuda.Event()
                arrived[p].record(up)
        total = 0
        for p in PARTS:
            stream.wait_event(arrived[p])
            g.part(p)  # returns after its results are complete (it reads their count)
            outs = results_of(p)
            done = torch.cuda.Event()
            done.record(stream)
            down.wait_event(done)
            with torch.cuda.stream(down):
                for i, o in enumerate(outs):
                    pinned_like((p, i), o).copy_(o, non_blocking=True)
                    o.record_stream(down)
            total += sum(o.numel() * o.element_size() for o in outs)
        down.synchronize()
        d2h[0] = total

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), world, stream.device)
    return {"value": whole_job_rate(rows_step, world, args.steps, ms), "unit": "rows/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h[0],
            "ms_per_step": ms / args.steps,
            "copies": "pipelined: inputs up on one stream, results down on another"}


if __name__ == "__main__":
    sys.exit(main())
