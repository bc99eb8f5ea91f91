"""The batched workload: thousands of uneven key/value group-bys and join
partitions, run (a) as one batch -- sizes from the learned planner (one
sketch launch and one network launch for all instances), then one memset and
two persistent launches replayed from a CUDA graph, with the autotuned tile
shape -- and (b) the plain way, one call sequence per instance (exact
pre-pass + aggregation per group-by; build, count and probe per join).

Both forms give the same groups and pairs; `compare` checks that instance by
instance.  Instances whose learned table overflowed are re-run exactly on
their own (the planner's fallback).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import rel

GB_OPS = ["sum", "count"]


def kv_query(keys: torch.Tensor, vals: torch.Tensor, ops=GB_OPS) -> dict:
    return {"cols": [keys, vals], "keys": [0], "preds": [], "aggs": [(op, 1, []) for op in ops]}


def learned_sizes(gb_inputs, planner_params: torch.Tensor | None = None):
    """Per group-by (est_groups, slots, variant) from the library's batched
    learned planning (rel_plan_size_batched: one sketch launch, one network
    launch, the learned sizing rule).  planner_params: FP32 network
    parameters to use instead of the registered ones (registered for the
    call, then the previous network is put back)."""
    if not gb_inputs:
        return []
    keys = [k for k, _ in gb_inputs]
    vals = [v for _, v in gb_inputs]
    if planner_params is None:
        plans = rel.plan_kv_batched(keys, vals, GB_OPS)
    else:
        prev = rel._planner_ref
        rel.planner_set(planner_params)
        try:
            plans = rel.plan_kv_batched(keys, vals, GB_OPS)
        finally:
            if prev is None:
                rel.planner_set(None)
            else:
                rel._planner_ref = prev
                rel.load().rel_planner_set(prev[1].data_ptr(), prev[0].data_ptr())
    return [(p.est_groups, p.slots, p.variant) for p in plans]


def make_batch(gb_inputs, join_inputs, sizes) -> rel.Batch:
    gs = []
    for (k, v), (est, slots, variant) in zip(gb_inputs, sizes):
        # est drives shared-memory placement; a network that prefers the
        # global table gets none
        gs.append({"keys": k, "vals": v, "ops": GB_OPS, "slots": slots,
                   "est_groups": est if variant == rel.VAR_SMEM else 1 << 40,
                   "capacity": max(1, min(k.numel(), slots))})
    js = [{"build_keys": bk, "build_payload": bp, "probe_keys": pk,
           "capacity": max(1, pk.numel())} for bk, bp, pk in join_inputs]
    return rel.Batch(gs, js)


def fallback(batch: rel.Batch, counts, flags):
    """Re-run, one by one, the instances the batch could not finish: a table
    overflow (group-by: exact re-plan) or an output larger than its capacity.
    Returns {index: outputs}."""
    ng = len(batch.gspec)
    redo = {}
    for i, f in enumerate(flags):
        if not f:
            continue
        if i < ng:
            q = batch.gspec[i]
            keys, aggs, _ = rel.groupby_auto(kv_query(q["keys"], q["vals"]), flags=rel.PLAN_EXACT)
            redo[i] = (keys, aggs)
        else:
            q = batch.jspec[i - ng]
            t = rel.JoinTable(q["build_keys"], q["build_payload"])
            redo[i] = t.probe(q["probe_keys"], capacity=max(1, t.count(q["probe_keys"])))
    return redo


def run_plain(gb_inputs, join_inputs):
    """One call sequence per instance; returns the outputs in order."""
    out = []
    for k, v in gb_inputs:
        keys, aggs, _ = rel.groupby_auto(kv_query(k, v), flags=rel.PLAN_EXACT, capacity=None)
        out.append((keys, aggs))
    for bk, bp, pk in join_inputs:
        t = rel.JoinTable(bk, bp)
        n = t.count(pk)
        out.append(t.probe(pk, capacity=max(1, n)))
    return out


def _same_groups(a, b) -> bool:
    (ka, aa), (kb, ab) = a, b
    if ka.numel() != kb.numel():
        return False
    sa, oa = torch.sort(ka)
    sb, ob = torch.sort(kb)
    return torch.equal(sa, sb) and all(torch.equal(x[oa], y[ob]) for x, y in zip(aa, ab))


def _same_pairs(a, b) -> bool:
    pa, ba, ya = a
    pb, bb, yb = b
    if pa.numel() != pb.numel():
        return False
    ka = pa.to(torch.int64) * (1 << 32) + ba.to(torch.int64)
    kb = pb.to(torch.int64) * (1 << 32) + bb.to(torch.int64)
    sa, oa = torch.sort(ka)
    sb, ob = torch.sort(kb)
    return torch.equal(sa, sb) and torch.equal(ya[oa], yb[ob])


def batch_outputs(batch: rel.Batch, counts, redo):
    ng = len(batch.gspec)
    out = []
    for i in range(ng + len(batch.jspec)):
        if i in redo:
            out.append(redo[i])
        elif i < ng:
            out.append(batch.groupby_output(i, counts[i]))
        else:
            out.append(batch.join_output(i - ng, counts[i]))
    return out


def compare(batched_out, plain_out, n_groupby: int) -> int:
    """Number of instances whose results differ."""
    bad = 0
    for i, (a, b) in enumerate(zip(batched_out, plain_out)):
        same = _same_groups(a, b) if i < n_groupby else _same_pairs(a, b)
        bad += not same
    return bad


def measure(gb_inputs, join_inputs, reps: int = 3, autotune: bool = True,
            candidates=None, planner_params=None) -> dict:
    """Wall time of both forms (inputs resident), results compared."""
    sync = torch.cuda.synchronize
    rows = sum(k.numel() for k, _ in gb_inputs) + sum(pk.numel() for _, _, pk in join_inputs)
    # batched: plan (sketch + network), prepare (+ autotune), graph, replay
    sync()
    t0 = time.perf_counter()
    sizes = learned_sizes(gb_inputs, planner_params)
    b = make_batch(gb_inputs, join_inputs, sizes)
    sync()
    t_plan = time.perf_counter() - t0
    tuned = None
    if autotune:
        tuned, _ = b.autotune(candidates)
    else:
        b.prepare()
    g = b.capture()
    times = []
    for _ in range(reps):
        sync()
        t0 = time.perf_counter()
        g.replay()
        counts, flags = b.results()
        redo = fallback(b, counts, flags)
        sync()
        times.append(time.perf_counter() - t0)
    t_batch = float(np.median(times))
    batched_out = batch_outputs(b, counts, redo)
    device = device_times(b, g, gb_inputs, join_inputs, counts)
    # plain
    times = []
    plain_out = None
    for _ in range(reps):
        sync()
        t0 = time.perf_counter()
        plain_out = run_plain(gb_inputs, join_inputs)
        sync()
        times.append(time.perf_counter() - t0)
    t_plain = float(np.median(times))
    mismatches = compare(batched_out, plain_out, len(gb_inputs))
    return {"instances": len(gb_inputs) + len(join_inputs), "rows": rows,
            "batched_s": t_batch, "plan_s": t_plan, "plain_s": t_plain,
            "batched_rows_per_s": rows / t_batch,
            "batched_with_plan_rows_per_s": rows / (t_batch + t_plan),
            "plain_rows_per_s": rows / t_plain, "speedup": t_plain / t_batch,
            "speedup_with_plan": t_plain / (t_batch + t_plan),
            "fallbacks": len(redo), "mismatches": mismatches, "config": tuned or b.config,
            "device": device}


def device_times(b: rel.Batch, graph, gb_inputs, join_inputs, counts) -> dict:
    """Device time of the graph replay alone (CUDA events, no read-back, no
    fallback re-runs) and of each persistent launch (one direct run with the
    library's launch timing), with their algorithmic bytes: launch A reads
    every group-by row (key + value) and every build row (key + payload);
    launch B reads every probe key and writes every pair (16 bytes) and every
    group (key + two aggregates)."""
    sync = torch.cuda.synchronize
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sync()
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    rel.profile_start()
    b.run()
    sync()
    kern = {}
    for name, t in rel.profile_stop():
        kern[name] = kern.get(name, 0.0) + t
    ng = len(gb_inputs)
    a_bytes = sum(k.numel() * (k.element_size() + 8) for k, _ in gb_inputs) + \
        sum(bk.numel() * 16 for bk, _, _ in join_inputs)
    b_bytes = sum(pk.numel() * 8 for _, _, pk in join_inputs) + \
        16 * sum(counts[ng:]) + 24 * sum(counts[:ng])
    out = {"replay_ms": float(np.median(ms)), "kernels_ms": kern,
           "batch_a_bytes": a_bytes, "batch_b_bytes": b_bytes}
    if kern.get("batch_a"):
        out["batch_a_gbs"] = a_bytes / (kern["batch_a"] / 1e3) / 1e9
    if kern.get("batch_b"):
        out["batch_b_gbs"] = b_bytes / (kern["batch_b"] / 1e3) / 1e9
    return out
