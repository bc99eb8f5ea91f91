"""The batched workload driver at toy scale: batched (learned sizes, graph
replay, autotuned) and plain forms agree instance by instance, and a sample
of instances matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import batched, rel
from synth import gpu as G

from gpu_util import canon_groupby, canon_join

pytestmark = pytest.mark.gpu


def small_inputs():
    r = G.batch_recipe(3, n_groupby=24, n_join=6)
    for i, x in enumerate(r["groupby"]):
        x["rows"] = max(1, x["rows"] // 40)
    for x in r["join"]:
        x["build"] = max(1, x["build"] // 20)
        x["probe"] = max(1, x["probe"] // 20)
    r["groupby"][0]["rows"] = 0  # an empty instance
    return G.batch_inputs(r)


def test_batched_equals_plain_and_oracle():
    gb, jn = small_inputs()
    params = torch.from_numpy(synth.mlp_params(9)).cuda()
    res = batched.measure(gb, jn, reps=1, autotune=True,
                          candidates=[(256, 8, 1, 512), (128, 4, 2, 0)], planner_params=params)
    assert res["mismatches"] == 0
    # and the plain form against the oracle on a sample
    for k, v in gb[:6]:
        q = oracle.kv_query(k.cpu().numpy(), v.cpu().numpy(), ops=("sum", "count"))
        ek, ea = oracle.groupby(q)
        keys, aggs, _ = rel.groupby_auto(batched.kv_query(k, v), flags=rel.PLAN_EXACT)
        gk, ga = canon_groupby(keys, aggs)
        assert np.array_equal(gk, ek) and np.array_equal(ga, ea)
    for bk, bp, pk in jn[:3]:
        e = oracle.join(bk.cpu().numpy(), bp.cpu().numpy(), pk.cpu().numpy())
        got = canon_join(*rel.JoinTable(bk, bp).probe(pk))
        assert all(np.array_equal(x, y) for x, y in zip(got, e))


def test_learned_underestimate_falls_back():
    gb, jn = small_inputs()
    p = np.zeros(rel.MLP_PARAMS, np.float32)  # y0 = 0: sample-sized tables
    sizes = batched.learned_sizes(gb, torch.from_numpy(p).cuda())
    b = batched.make_batch(gb, jn, sizes).prepare()
    b.run()
    counts, flags = b.results()
    redo = batched.fallback(b, counts, flags)
    out = batched.batch_outputs(b, counts, redo)
    plain = batched.run_plain(gb, jn)
    assert batched.compare(out, plain, len(gb)) == 0
