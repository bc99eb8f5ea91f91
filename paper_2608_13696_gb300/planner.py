"""The learned planner's data, training and evaluation driver.

  collect  -- run seeded group-by instances (GPU-generated key/value columns,
              see synth/gpu.py) through the library and record, per run, the
              sketch's 264 features, log2 of the exact number of groups (the
              exact pre-pass) and the device time of each variant (per-CTA
              tables, global table, partitioned) sized from the exact count,
              median of `reps` runs with L2 flushed before each; the label is
              the fastest variant.
  train    -- fit the planner network on collected runs with the library's
              own kernels (rel_mlp_forward / rel_mlp_backward / rel_mlp_adamw):
              loss = (y0 - log2 groups)^2 + cross-entropy(variant), AdamW,
              FP32 master weights with a BF16 copy; checkpoints every epoch and
              resumes from the last one.
  evaluate -- on instances with unseen seeds: the learned plan against the
              exact pre-pass plan and against sizing for n_rows groups, all
              through rel_groupby_auto, results compared bit for bit (keys and
              aggregates after sorting), wall time per instance with inputs
              resident and L2 flushed.

    python -m paper_2608_13696_gb300.planner collect --seeds 0:8000 --out runs.npz
    python -m paper_2608_13696_gb300.planner train runs.npz --out weights.npz
    python -m paper_2608_13696_gb300.planner evaluate --seeds 1000000:1002000 --weights weights.npz

Everything on the data path runs in librel's kernels; torch supplies device
memory, streams, events and batch indexing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import rel

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "planner_weights.npz")
VARIANTS = (rel.VAR_SMEM, rel.VAR_GLOBAL, rel.VAR_PARTITIONED)
L2_FLUSH_BYTES = 256 << 20


def kv_query(keys: torch.Tensor, vals: torch.Tensor) -> dict:
    """sum, count, min, max of vals grouped by keys."""
    return {"cols": [keys, vals], "keys": [0], "preds": [],
            "aggs": [("sum", 1, []), ("count", 1, []), ("min", 1, []), ("max", 1, [])]}


def _parse_range(s: str) -> range:
    a, b = s.split(":")
    return range(int(a), int(b))


class _Flush:
    def __init__(self, device):
        self.buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)

    def __call__(self):
        self.buf.fill_(1)


def _time_plan(qc, plan, reps, flush, ws, cap, give_up_ms=float("inf")):
    """Median device time of `reps` runs; stops after the first run when that
    one is already slower than give_up_ms (it cannot be the fastest)."""
    times = []
    for r in range(reps):
        if r == 1 and times[0] > give_up_ms:
            break
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rel.groupby(qc, plan=plan, capacity=cap, ws=ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


# share of the runs that are filtered, packed-key inputs (the lineitem shape:
# date filter of varying selectivity, (flag, status) key, five aggregates)
LINEITEM_SHARE = 0.05
LINEITEM_ROWS = (1_000_000, 20_000_000)


def _lineitem_instance(seed: int, dev):
    """A filtered packed-key run: lineitem-like columns (host generator) of
    log-uniform rows, keeping date <= a seeded threshold."""
    import synth
    from . import workloads

    rng = np.random.default_rng(seed)
    lo, hi = LINEITEM_ROWS
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    li = synth.lineitem(n, seed=seed)
    q = workloads.lineitem_query(li, date_hi=int(rng.integers(100, 2527)))
    q["cols"] = [torch.from_numpy(c).to(dev) for c in q["cols"]]
    return q, {"rows": n, "domain": 6, "fam": 9, "s": 0.0}


def _is_lineitem(seed: int) -> bool:
    return np.random.default_rng((seed, 7)).random() < LINEITEM_SHARE


def collect(seeds, out: str, reps: int = 3, rows_lo: int = 1_000_000,
            rows_hi: int = 50_000_000, log_every: int = 200, save_every: int = 2000,
            with_lineitem: bool = False) -> dict:
    from synth import gpu as G

    dev = torch.device("cuda")
    flush = _Flush(dev)
    feats, t_ndv, label, times, meta = [], [], [], [], []
    ws = None
    t_start = time.time()
    for i, seed in enumerate(seeds):
        if with_lineitem and _is_lineitem(seed):
            qc, inst = _lineitem_instance(seed, dev)
            k = v = None
        else:
            inst = G.instance(seed, rows_lo=rows_lo, rows_hi=rows_hi)
            k, v = G.instance_kv(inst, dev)
            qc = kv_query(k, v)
        n_aggs = len(qc["aggs"])
        s = rel.sketch(qc)
        exact = rel.plan_groupby(qc, flags=rel.PLAN_EXACT)
        ndv = max(1, int(exact.est_groups))
        row = []
        for var in VARIANTS:
            try:
                plan = rel.plan_groupby(qc, flags=rel.PLAN_SKETCH | rel.plan_force(var),
                                        groups_hint=ndv)
            except rel.RelError as e:  # e.g. no partitioned variant for packed keys
                if e.status != rel.REL_E_UNSUPPORTED:
                    raise
                row.append(float("inf"))
                continue
            need = int(rel.load().rel_plan_ws_bytes(plan, n_aggs, inst["rows"]))
            if ws is None or ws.numel() < need:
                ws = None
                torch.cuda.empty_cache()
                ws = torch.empty(need, dtype=torch.uint8, device=dev)
            try:
                best = min(row) if row else float("inf")
                row.append(_time_plan(qc, plan, reps, flush, ws, ndv + 1, give_up_ms=2 * best))
            except rel.RelError as e:  # a variant that cannot run on this input
                if e.status not in (rel.REL_E_OVERFLOW, rel.REL_E_UNSUPPORTED):
                    raise
                print(f"collect: seed {seed} variant {var}: {e}", file=sys.stderr)
                row.append(float("inf"))
        feats.append(np.frombuffer(bytes(s.features), dtype=np.float32).copy())
        t_ndv.append(math.log2(ndv))
        label.append(int(np.argmin(row)))
        times.append(row)
        meta.append((seed, inst["rows"], inst["domain"], inst["fam"], inst["s"], ndv))
        del k, v, qc
        if log_every and (i + 1) % log_every == 0:
            print(f"collect: {i + 1} runs, {time.time() - t_start:.0f} s", file=sys.stderr)
        if save_every and (i + 1) % save_every == 0:
            _save_runs(out, feats, t_ndv, label, times, meta)
    return _save_runs(out, feats, t_ndv, label, times, meta)


def _save_runs(out, feats, t_ndv, label, times, meta) -> dict:
    data = {"features": np.array(feats, np.float32).reshape(-1, rel.MLP_IN),
            "log2_groups": np.array(t_ndv, np.float32), "label": np.array(label, np.int32),
            "times_ms": np.array(times, np.float32).reshape(-1, 3),
            "meta": np.array(meta, np.float64).reshape(-1, 6)}
    np.savez_compressed(out, **data)
    return data


def init_params(seed: int) -> np.ndarray:
    """Weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases; output 0's
    bias starts at 10 (log2 of a middling group count)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fo, fi in ((rel.MLP_HIDDEN, rel.MLP_IN), (rel.MLP_HIDDEN, rel.MLP_HIDDEN),
                   (rel.MLP_OUT, rel.MLP_HIDDEN)):
        s = 1.0 / math.sqrt(fi)
        parts += [rng.uniform(-s, s, fo * fi), np.zeros(fo)]
    p = np.concatenate(parts).astype(np.float32)
    p[-rel.MLP_OUT] = 10.0
    return p


def _load_runs(paths):
    parts = [np.load(p) for p in paths]
    return {k: np.concatenate([d[k] for d in parts]) for k in parts[0].files}


def metrics(y: np.ndarray, data: dict, idx: np.ndarray) -> dict:
    """Log2-size error, variant accuracy and misprediction rate (chosen
    variant more than 5 % slower than the fastest measured)."""
    err = y[:, 0] - data["log2_groups"][idx]
    choice = np.argmax(y[:, 1:], axis=1)
    t = data["times_ms"][idx]
    chosen = t[np.arange(len(idx)), choice]
    return {"n": int(len(idx)), "log2_mae": float(np.mean(np.abs(err))),
            "log2_p95": float(np.percentile(np.abs(err), 95)),
            "under_1.25x": float(np.mean(2.0 ** y[:, 0] * 1.25 < 2.0 ** data["log2_groups"][idx])),
            "variant_acc": float(np.mean(choice == data["label"][idx])),
            "mispredict": float(np.mean(chosen > 1.05 * t.min(axis=1))),
            "time_chosen_over_best": float(chosen.sum() / t.min(axis=1).sum())}


def train(paths, out: str, epochs: int = 20, batch: int = 256, lr: float = 1e-3,
          wd: float = 1e-4, val_frac: float = 0.1, seed: int = 0, ckpt: str | None = None) -> dict:
    data = _load_runs(paths)
    dev = torch.device("cuda")
    N = len(data["label"])
    order = np.random.default_rng(seed).permutation(N)
    n_val = max(1, int(N * val_frac))
    val_idx, tr_idx = np.sort(order[:n_val]), order[n_val:]
    X = torch.from_numpy(data["features"]).to(dev)
    T = torch.from_numpy(data["log2_groups"]).to(dev)
    V = torch.from_numpy(data["label"]).to(dev)
    p = torch.from_numpy(init_params(seed)).to(dev)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    step, epoch0 = 0, 0
    if ckpt and os.path.exists(ckpt):
        c = np.load(ckpt)
        p.copy_(torch.from_numpy(c["params"]))
        m.copy_(torch.from_numpy(c["m"]))
        v.copy_(torch.from_numpy(c["v"]))
        step, epoch0 = int(c["step"]), int(c["epoch"])
    bf = torch.empty(rel.MLP_PARAMS, dtype=torch.bfloat16, device=dev)
    rel.mlp_round(p, bf)
    acts = torch.empty((batch, 2 * rel.MLP_HIDDEN), device=dev)
    grad = torch.empty_like(p)
    loss = torch.empty(1, device=dev)
    ws = torch.empty(int(rel.load().rel_mlp_ws_bytes(batch)), dtype=torch.uint8, device=dev)
    history = []
    for epoch in range(epoch0, epochs):
        perm = np.random.default_rng((seed, epoch)).permutation(tr_idx)
        tot, nb = 0.0, 0
        for b0 in range(0, len(perm) - batch + 1, batch):
            ib = torch.from_numpy(perm[b0:b0 + batch]).to(dev)
            xb, tb, vb = X[ib].contiguous(), T[ib].contiguous(), V[ib].contiguous()
            y = rel.mlp_forward(bf, p, xb, acts)
            rel.mlp_backward(bf, xb, acts, y, tb, vb, grad, loss, ws=ws)
            step += 1
            rel.mlp_adamw(p, bf, m, v, grad, step, lr=lr, weight_decay=wd)
            tot += float(loss.item())
            nb += 1
        yv = rel.mlp_forward(bf, p, X[torch.from_numpy(val_idx).to(dev)].contiguous())
        mv = metrics(yv.cpu().numpy(), data, val_idx)
        mv.update(epoch=epoch + 1, train_loss=tot / max(1, nb))
        history.append(mv)
        print("train:", json.dumps(mv), file=sys.stderr)
        if ckpt:
            np.savez(ckpt, params=p.cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(),
                     step=step, epoch=epoch + 1)
    info = {"runs": int(N), "train": int(len(tr_idx)), "val": int(n_val), "epochs": epochs,
            "batch": batch, "lr": lr, "weight_decay": wd, "seed": seed,
            "val_metrics": history[-1] if history else None}
    np.savez(out, params=p.cpu().numpy(), info=json.dumps(info))
    return info


def load_weights(path: str = DEFAULT_WEIGHTS) -> torch.Tensor:
    w = np.load(path)
    return torch.from_numpy(w["params"].astype(np.float32))


def use_default(device="cuda") -> None:
    """Register the committed trained network for REL_PLAN_LEARNED."""
    rel.planner_set(load_weights().to(device))


def _sorted(keys, aggs):
    k, o = torch.sort(keys)
    return k, [a[o] for a in aggs]


def evaluate(seeds, weights: str = DEFAULT_WEIGHTS, rows_lo: int = 1_000_000,
             rows_hi: int = 50_000_000, with_labels: bool = True, log_every: int = 200,
             with_rows: bool = True) -> dict:
    """The learned plan vs the exact pre-pass (and, with_rows, vs sizing for
    n_rows)."""
    from synth import gpu as G

    dev = torch.device("cuda")
    rel.planner_set(load_weights(weights).to(dev))
    flush = _Flush(dev)
    ws = None
    forms = {"learned": rel.PLAN_LEARNED | rel.PLAN_SKETCH,
             "exact": rel.PLAN_EXACT | rel.PLAN_SKETCH}
    if with_rows:
        forms["rows"] = rel.PLAN_SKETCH
    tot = {f: 0.0 for f in forms}
    rows_total = 0
    mismatches, fallbacks = 0, 0
    per = []
    for i, seed in enumerate(seeds):
        inst = G.instance(seed, rows_lo=rows_lo, rows_hi=rows_hi)
        k, v = G.instance_kv(inst, dev)
        qc = kv_query(k, v)
        need = rel.auto_ws_bytes(qc)
        if ws is None or ws.numel() < need:
            ws = None
            torch.cuda.empty_cache()
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        res, ms = {}, {}
        for f, flags in forms.items():
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            keys, aggs, plan = rel.groupby_auto(qc, flags=flags, ws=ws)
            torch.cuda.synchronize()
            ms[f] = (time.perf_counter() - t0) * 1e3
            tot[f] += ms[f]
            res[f] = (_sorted(keys, aggs), plan)
            if f == "learned" and plan.flags & rel.PLAN_FELL_BACK:
                fallbacks += 1
        (ke, ae), pe = res["exact"]
        for f in forms:
            if f == "exact":
                continue
            (kf, af), _ = res[f]
            if not (torch.equal(kf, ke) and all(torch.equal(x, y) for x, y in zip(af, ae))):
                mismatches += 1
        rec = {"seed": seed, "rows": inst["rows"], "family": inst["family"],
               "domain": inst["domain"], "groups": int(pe.est_groups),
               "est_learned": int(res["learned"][1].est_groups),
               "variant_learned": int(res["learned"][1].variant),
               "fell_back": bool(res["learned"][1].flags & rel.PLAN_FELL_BACK), **ms}
        if with_labels:
            t = []
            for var in VARIANTS:
                plan = rel.plan_groupby(qc, flags=rel.PLAN_SKETCH | rel.plan_force(var),
                                        groups_hint=max(1, rec["groups"]))
                t.append(_time_plan(qc, plan, 1, flush, ws, rec["groups"] + 1))
            rec["variant_ms"] = t
        per.append(rec)
        rows_total += inst["rows"]
        del k, v, qc, res
        if log_every and (i + 1) % log_every == 0:
            print(f"evaluate: {i + 1} instances", file=sys.stderr)
    out = {"instances": len(per), "rows": rows_total, "mismatches": mismatches,
           "fallbacks": fallbacks,
           "ms_total": tot, "speedup_vs_exact": tot["exact"] / tot["learned"],
           "rows_per_s": {f: rows_total / (tot[f] * 1e-3) for f in forms}}
    if with_rows:
        out["speedup_vs_rows"] = tot["rows"] / tot["learned"]
    if with_labels and per:
        err = np.array([math.log2(max(1, r["est_learned"]) / 1.25) - math.log2(max(1, r["groups"]))
                        for r in per])
        vt = np.array([r["variant_ms"] for r in per])
        ch = np.array([VARIANTS.index(r["variant_learned"]) if r["variant_learned"] in VARIANTS
                       else 1 for r in per])
        chosen = vt[np.arange(len(per)), ch]
        out.update(log2_mae=float(np.mean(np.abs(err))),
                   mispredict=float(np.mean(chosen > 1.05 * vt.min(axis=1))),
                   variant_time_over_best=float(chosen.sum() / vt.min(axis=1).sum()))
    out["per_instance"] = per
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2608_13696_gb300.planner")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--seeds", default="0:1000")
    c.add_argument("--out", required=True)
    c.add_argument("--reps", type=int, default=3)
    c.add_argument("--rows-lo", type=int, default=1_000_000)
    c.add_argument("--rows-hi", type=int, default=50_000_000)
    c.add_argument("--with-lineitem", action="store_true",
                   help="make about 5 %% of the runs filtered packed-key (lineitem-like) inputs")
    t = sub.add_parser("train")
    t.add_argument("runs", nargs="+")
    t.add_argument("--out", required=True)
    t.add_argument("--epochs", type=int, default=20)
    t.add_argument("--batch", type=int, default=256)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--wd", type=float, default=1e-4)
    t.add_argument("--seed", type=int, default=0)
    t.add_argument("--ckpt", default=None)
    e = sub.add_parser("evaluate")
    e.add_argument("--seeds", default="1000000:1002000")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--rows-lo", type=int, default=1_000_000)
    e.add_argument("--rows-hi", type=int, default=50_000_000)
    e.add_argument("--no-labels", action="store_true")
    e.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.cmd == "collect":
        collect(_parse_range(a.seeds), a.out, reps=a.reps, rows_lo=a.rows_lo, rows_hi=a.rows_hi,
                with_lineitem=a.with_lineitem)
    elif a.cmd == "train":
        print(json.dumps(train(a.runs, a.out, epochs=a.epochs, batch=a.batch, lr=a.lr, wd=a.wd,
                               seed=a.seed, ckpt=a.ckpt)))
    else:
        r = evaluate(_parse_range(a.seeds), a.weights, rows_lo=a.rows_lo, rows_hi=a.rows_hi,
                     with_labels=not a.no_labels)
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        r.pop("per_instance")
        print(json.dumps(r))


if __name__ == "__main__":
    main()
