"""The planner and batched workloads checked against the CPU oracle on
seeded instances (the bench compares every instance with the plain GPU form;
these compare with the oracle): 32 planner-workload instances of up to 5e6
rows through the learned plan with the committed network, and a 48-group-by
+ 8-partition slice of the batched workload through one graph-replayed
batch."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2608_13696_gb300 import batched, planner, rel
from synth import gpu as G

from gpu_util import canon_groupby, canon_join

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(not os.path.exists(planner.DEFAULT_WEIGHTS), reason="no trained network")
@pytest.mark.parametrize("seed", range(3_000_000, 3_000_032))
def test_planner_instance_matches_oracle(seed):
    planner.use_default()
    inst = G.instance(seed, rows_lo=100_000, rows_hi=5_000_000)
    k, v = G.instance_kv(inst)
    keys, aggs, plan = rel.groupby_auto(planner.kv_query(k, v),
                                        flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH)
    ek, ea = oracle.groupby(oracle.kv_query(k.cpu().numpy(), v.cpu().numpy()))
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, ek) and np.array_equal(ga, ea), inst


@pytest.mark.skipif(not os.path.exists(planner.DEFAULT_WEIGHTS), reason="no trained network")
def test_batched_slice_matches_oracle():
    planner.use_default()
    r = G.batch_recipe(7)
    r["groupby"] = [dict(x, rows=min(x["rows"], 2_000_000)) for x in r["groupby"][:48]]
    r["join"] = [dict(x, probe=min(x["probe"], 2_000_000)) for x in r["join"][:8]]
    gb, jn = G.batch_inputs(r)
    b = batched.make_batch(gb, jn, batched.learned_sizes(gb))
    b.autotune([(256, 8, 1, 512), (512, 4, 1, 512)], reps=1)
    g = b.capture()
    g.replay()
    counts, flags = b.results()
    redo = batched.fallback(b, counts, flags)
    out = batched.batch_outputs(b, counts, redo)
    for i, (k, v) in enumerate(gb):
        ek, ea = oracle.groupby(oracle.kv_query(k.cpu().numpy(), v.cpu().numpy(),
                                                ops=("sum", "count")))
        gk, ga = canon_groupby(*out[i])
        assert np.array_equal(gk, ek) and np.array_equal(ga, ea), i
    for i, (bk, bp, pk) in enumerate(jn):
        e = oracle.join(bk.cpu().numpy(), bp.cpu().numpy(), pk.cpu().numpy())
        got = canon_join(*out[len(gb) + i])
        assert all(np.array_equal(x, y) for x, y in zip(got, e)), i
