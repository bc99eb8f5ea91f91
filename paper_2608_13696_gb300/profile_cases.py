"""Small cases of the hot kernels, one launch each, for profiler captures.

    python -m paper_2608_13696_gb300.profile_cases

runs, on 5e7-row inputs: the exact distinct-count pre-pass and a partitioned
group-by with the sample sketch over Zipf(1.1) key/value rows; a streaming
group-by with pinned keys over four-key rows; a join table of 1e6 keys probed
with 4e6 keys.  Small enough for a full-section capture of each launch.
"""
from __future__ import annotations

import sys

import torch

from . import rel


def kv_query(k, v):
    return {"cols": [k, v], "keys": [0], "preds": [],
            "aggs": [("sum", 1, []), ("count", 1, []), ("min", 1, []), ("max", 1, [])]}


def main(n: int = 50_000_000) -> None:
    import synth

    zk, zv = synth.zipf_kv(n, seed=0)
    q = kv_query(torch.from_numpy(zk).cuda(), torch.from_numpy(zv).cuda())
    del zk, zv
    ex = rel.plan_groupby(q, flags=rel.PLAN_EXACT)
    p = rel.plan_groupby(q, flags=rel.plan_force(rel.VAR_PARTITIONED) | rel.PLAN_SKETCH,
                         groups_hint=ex.est_groups)
    rel.groupby(q, plan=p, capacity=ex.est_groups + 1)
    fk, fv = synth.few_keys_kv(n, n_keys=4, seed=0)
    q4 = kv_query(torch.from_numpy(fk).cuda(), torch.from_numpy(fv).cuda())
    p4 = rel.plan_groupby(q4, flags=rel.PLAN_SKETCH | rel.plan_force(rel.VAR_GLOBAL), groups_hint=4)
    rel.groupby(q4, plan=p4, capacity=8)
    bk, bp = synth.join_build(1_000_000, seed=0)
    pk, _ = synth.join_probe(4_000_000, 1_000_000, seed=0)
    t = rel.JoinTable(torch.from_numpy(bk).cuda(), torch.from_numpy(bp).cuda())
    t.probe(torch.from_numpy(pk).cuda(), capacity=4_000_000)
    torch.cuda.synchronize()
    print("ok", ex.est_groups)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 50_000_000)
