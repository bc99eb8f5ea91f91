"""Small cases of the library's kernels for profiler captures, one case per
run, each launching the kernels of interest a few times at most.

    python -m paper_2608_13696_gb300.profile_cases CASE

CASE (inputs seeded and synthetic, as in the bench):
  distinct  exact distinct count of 5e7 Zipf(1.1) keys (distinct_k)
  part      partitioned group-by of 5e7 Zipf(1.1) key/value rows with the
            sample sketch's pins (histogram, scan, two scatter levels,
            aggregation, compaction)
  stream    streaming group-by of 5e7 four-key rows with pinned keys (gb_stream)
  join      join build of 1e6 unique keys and probe of 1.6e7 keys (90 % hits)
  lineitem  fused filter + group-by of 2e7 lineitem rows: exact count (staged
            key set), sketch, aggregation in thread-private shared words,
            compaction
  mlp       planner network forward, backward and AdamW on a batch of 256
  batch     a batch of 512 group-bys and 64 join partitions (the batched
            workload's recipe, rows divided by 8): the two persistent launches
  shard     owner split of 2e6 partial groups over 8 ranks
  hll       full-data HyperLogLog of 5e7 Zipf(1.1) keys
Sizes keep every case below a few GB of device memory, with inputs above the
129 MB L2 where the kernel streams.  Algorithmic bytes: inputs read once and
outputs written once (16-byte records for the partition passes, 16 bytes
per match for the join probe); hash-table and workspace traffic excluded.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from . import rel


def kv_query(k, v, ops=("sum", "count", "min", "max")):
    return {"cols": [k, v], "keys": [0], "preds": [], "aggs": [(o, 1, []) for o in ops]}


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case_distinct(n=50_000_000):
    import synth

    zk, zv = synth.zipf_kv(n, seed=0)
    q = kv_query(_cuda(zk), _cuda(zv), ops=("count",))
    rel.plan_groupby(q, flags=rel.PLAN_EXACT)
    return {"gb_main_keyset": (n, "rows", 8 * n)}


def case_part(n=50_000_000):
    import synth

    zk, zv = synth.zipf_kv(n, seed=0)
    q = kv_query(_cuda(zk), _cuda(zv))
    p = rel.plan_groupby(q, flags=rel.plan_force(rel.VAR_PARTITIONED) | rel.PLAN_SKETCH,
                         groups_hint=3_300_000)
    k, aggs = rel.groupby(q, plan=p, capacity=4_000_000)
    kd = q["cols"][0]
    hot = torch.tensor([p.hot_keys[i] for i in range(p.n_hot)] + [-(1 << 63)], dtype=torch.int64,
                       device=kd.device)
    recs = int(n - torch.isin(kd, hot).sum().item())  # rows written as partition records
    out = k.numel() * 8 * (1 + len(aggs))
    return {"gb_part_hist": (n, "rows", 8 * n), "gb_part_scatter": (n, "rows", 16 * n + 16 * recs),
            "gb_part_l2": (n, "rows", 32 * recs),
            "gb_part_scan": (n, "rows", None), "gb_part_agg": (n, "rows", 16 * recs + out),
            "gb_compact": (n, "rows", out), "records": recs, "groups": k.numel()}


def case_stream(n=50_000_000):
    import synth

    fk, fv = synth.few_keys_kv(n, n_keys=4, seed=0)
    q = kv_query(_cuda(fk), _cuda(fv))
    p = rel.plan_groupby(q, flags=rel.PLAN_SKETCH, groups_hint=4)
    rel.groupby(q, plan=p, capacity=8)
    return {"gb_stream": (n, "rows", 16 * n)}


def case_join(nb=1_000_000, np_=16_000_000):
    import synth

    bk, bp = synth.join_build(nb, seed=0)
    pk, _ = synth.join_probe(np_, nb, seed=0)
    t = rel.JoinTable(_cuda(bk), _cuda(bp))
    m = t.probe(_cuda(pk), capacity=np_)[0].numel()
    return {"join_build": (nb, "build rows", 16 * nb), "join_probe": (np_, "probes", 8 * np_ + 16 * m),
            "matches": m}


def case_lineitem(n=20_000_000):
    import synth

    from .workloads import lineitem_query

    q = lineitem_query(synth.lineitem(n, seed=0))
    q["cols"] = [_cuda(c) for c in q["cols"]]
    p = rel.plan_groupby(q, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    rel.groupby(q, plan=p)
    used = set(q["keys"]) | {c[0] for c in q.get("preds", [])}
    return {"gb_main_staged_keyset": (n, "rows", sum(q["cols"][c].nbytes for c in used)),
            "gb_main_layered": (n, "rows", sum(c.nbytes for c in q["cols"])),
            "sketch": (1, "sketch", None)}


def case_mlp(batch=256):
    g = torch.Generator().manual_seed(0)
    p = (torch.rand(rel.MLP_PARAMS, generator=g) * 0.2 - 0.1).cuda()
    x = torch.rand(batch, rel.MLP_IN, generator=g).cuda()
    bf = torch.empty(rel.MLP_PARAMS, dtype=torch.bfloat16, device="cuda")
    rel.mlp_round(p, bf)
    acts = torch.empty((batch, 2 * rel.MLP_HIDDEN), device="cuda")
    y = rel.mlp_forward(bf, p, x, acts)
    t = torch.rand(batch, generator=g).cuda() * 20
    v = torch.randint(0, 3, (batch,), generator=g, dtype=torch.int32).cuda()
    grad = torch.empty_like(p)
    loss = torch.empty(1, device="cuda")
    rel.mlp_backward(bf, x, acts, y, t, v, grad, loss)
    m, s = torch.zeros_like(p), torch.zeros_like(p)
    rel.mlp_adamw(p, bf, m, s, grad, 1)
    return {"mlp_forward": (batch, "samples", None), "mlp_backward": (batch, "samples", None),
            "mlp_adamw": (rel.MLP_PARAMS, "parameters", None), "loss": float(loss.item())}


def case_batch():
    from synth import gpu as G

    from . import batched

    r = G.batch_recipe(0, n_groupby=512, n_join=64)
    for x in r["groupby"]:
        x["rows"] = max(1, x["rows"] // 8)
    for x in r["join"]:
        x["probe"] = max(1, x["probe"] // 8)
    gb, jn = G.batch_inputs(r)
    est = [min(k.numel(), 100_000) for k, _ in gb]
    sizes = [(e, 1 << max(4, (2 * e - 1).bit_length()),
              rel.VAR_SMEM if e <= 512 else rel.VAR_GLOBAL) for e in est]
    b = batched.make_batch(gb, jn, sizes).prepare((512, 4, 1, 512))
    b.run()
    b.results()
    rows = sum(k.numel() for k, _ in gb)
    gb_bytes = sum(k.nbytes + v.nbytes for k, v in gb)
    probes = sum(x[2].numel() for x in jn)
    jn_bytes = sum(sum(t.nbytes for t in x) for x in jn)
    return {"batch_a": (rows + probes, "rows", gb_bytes + jn_bytes),
            "batch_b": (rows + probes, "rows", None)}


def case_shard(n=2_000_000, world=8):
    g = torch.Generator().manual_seed(0)
    k = torch.randint(-(1 << 62), 1 << 62, (n,), generator=g).cuda()
    w = [torch.randint(-1000, 1000, (n,), generator=g).cuda() for _ in range(4)]
    rel.shard_split(k, w, world)
    return {"shard_scatter": (n, "groups", 2 * 8 * 5 * n)}


def case_hll(n=50_000_000):
    import synth

    zk, _ = synth.zipf_kv(n, seed=0)
    rel.key_hll(_cuda(zk))
    return {"hll": (n, "rows", 8 * n)}


CASES = {"distinct": case_distinct, "part": case_part, "stream": case_stream,
         "join": case_join, "lineitem": case_lineitem, "mlp": case_mlp, "batch": case_batch,
         "shard": case_shard, "hll": case_hll}


def main(argv) -> None:
    """Runs the named cases; prints per case one line `NAME ok JSON`, the
    JSON mapping each kernel id to [units, unit name, algorithmic bytes or
    null] for the summary of its capture."""
    import json

    rel.load()
    for name in argv or list(CASES):
        out = CASES[name]()
        torch.cuda.synchronize()
        print(name, "ok", json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1:])
