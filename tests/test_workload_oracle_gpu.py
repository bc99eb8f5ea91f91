"""The planner and batched workloads checked against the CPU oracle on
seeded instances (the bench compares every instance with the plain GPU form;
these compare with the oracle):
  * 32 planner-workload instances drawn over the workload's whole row range
    (1e6..5e7 rows, every key family), through the learned plan with the
    committed network and its exact fallback;
  * the full batched workload the bench runs (4096 group-bys + 512 join
    partitions, one graph-replayed batch with learned sizes and the
    autotuner): every instance of at most 2e6 rows, plus 32 seeded ones of the
    larger group-bys.
Large references run on hash partitions of the rows (oracle.partitioned) and
the many small ones on a thread pool (the oracle's C calls release the GIL)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from oracle import partitioned
from paper_2608_13696_gb300 import batched, planner, rel
from synth import gpu as G

from gpu_util import canon_groupby, canon_join

pytestmark = pytest.mark.gpu

needs_net = pytest.mark.skipif(not os.path.exists(planner.DEFAULT_WEIGHTS),
                               reason="no trained network")


@needs_net
@pytest.mark.parametrize("seed", range(3_000_000, 3_000_032))
def test_planner_instance_matches_oracle(seed):
    planner.use_default()
    inst = G.instance(seed, rows_lo=1_000_000, rows_hi=50_000_000)
    k, v = G.instance_kv(inst)
    keys, aggs, plan = rel.groupby_auto(planner.kv_query(k, v),
                                        flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH)
    ek, ea = partitioned.groupby(oracle.kv_query(k.cpu().numpy(), v.cpu().numpy()), sort=True)
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, ek) and np.array_equal(ga, ea), inst


@needs_net
def test_full_batched_workload_matches_oracle():
    planner.use_default()
    recipe = G.batch_recipe(0)
    gb, jn = G.batch_inputs(recipe)
    b = batched.make_batch(gb, jn, batched.learned_sizes(gb))
    b.autotune([c for c in rel.BATCH_SEARCH if c[2] in (1, 2)])
    g = b.capture()
    g.replay()
    counts, flags = b.results()
    redo = batched.fallback(b, counts, flags)
    out = batched.batch_outputs(b, counts, redo)
    torch.cuda.synchronize()
    small = [i for i, (k, _) in enumerate(gb) if k.numel() <= 2_000_000]
    large = [i for i, (k, _) in enumerate(gb) if k.numel() > 2_000_000]
    rng = np.random.default_rng(0)
    picked = sorted(small + list(rng.choice(large, size=min(32, len(large)), replace=False)))
    assert len(small) > 3000 and len(picked) >= len(small) + 32

    host_gb = {i: (gb[i][0].cpu().numpy(), gb[i][1].cpu().numpy()) for i in picked}
    host_jn = [tuple(t.cpu().numpy() for t in x) for x in jn]
    assert all(len(x[2]) <= 2_000_000 for x in host_jn)  # every join partition is checked

    def ref_gb(i):
        k, v = host_gb[i]
        return oracle.groupby(oracle.kv_query(k, v, ops=("sum", "count")))

    def ref_jn(j):
        return oracle.join(*host_jn[j])

    with ThreadPoolExecutor(max_workers=partitioned.default_threads()) as pool:
        refs_gb = dict(zip(picked, pool.map(ref_gb, picked)))
        refs_jn = list(pool.map(ref_jn, range(len(jn))))
    bad = []
    for i in picked:
        ek, ea = refs_gb[i]
        gk, ga = canon_groupby(*out[i])
        if not (np.array_equal(gk, ek) and np.array_equal(ga, ea)):
            bad.append(("groupby", i))
    for j, e in enumerate(refs_jn):
        got = canon_join(*out[len(gb) + j])
        if not all(np.array_equal(x, y) for x, y in zip(got, e)):
            bad.append(("join", j))
    assert not bad, bad[:10]
