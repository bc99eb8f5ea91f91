"""GPU parity of the sample sketch (rel_sketch) against the oracle's sketch --
integer fields bit-exact, features to float32 rounding -- and of group-bys
planned from it (hot keys pinned in thread-private slots) against the oracle
group-by."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, cuda, query_to_cuda

pytestmark = pytest.mark.gpu


def cases():
    li = synth.lineitem(250_000, seed=3)
    zk, zv = synth.zipf_kv(500_000, seed=4, n_ranks=100_000)
    fk, fv = synth.few_keys_kv(300_000, n_keys=4, seed=5)
    k32 = synth.uniform(50_000, -7, 7, seed=6, tag=3, dtype=np.int32)
    runs = np.repeat(np.arange(127, dtype=np.int64), 64)
    sent = np.array([np.iinfo(np.int64).min] * 10 + list(range(90)), dtype=np.int64)
    return {
        "lineitem": oracle.lineitem_query(li),
        "zipf": oracle.kv_query(zk, zv),
        "four": oracle.kv_query(fk, fv),
        "int32": oracle.kv_query(k32, zv[:50_000]),
        "runs": oracle.kv_query(runs, runs),
        "tiny_n": oracle.kv_query(zk[:37], zv[:37]),
        "sentinel": oracle.kv_query(sent, sent),
        "filtered_out": oracle.lineitem_query(synth.lineitem(9000, seed=7), date_hi=-1),
    }


CASES = cases()


@pytest.mark.parametrize("name", list(CASES))
def test_sketch_matches_oracle(name):
    q = CASES[name]
    s = rel.sketch(query_to_cuda(q))
    e = oracle.sketch(q)
    for f in ("sample_rows", "kept", "ndv", "singletons", "runs", "key_min", "key_max",
              "key_bits"):
        assert getattr(s, f) == e[f], f
    assert list(s.top_key) == e["top_key"].tolist()
    assert list(s.top_count) == e["top_count"].tolist()
    assert bytes(s.hll) == e["hll"].tobytes()
    np.testing.assert_allclose(np.array(s.features, dtype=np.float64), e["features"],
                               rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("name", ["lineitem", "zipf", "four", "int32", "sentinel", "runs"])
@pytest.mark.parametrize("flags", [rel.PLAN_EXACT | rel.PLAN_SKETCH, rel.PLAN_SKETCH])
def test_sketch_planned_groupby(name, flags):
    q = CASES[name]
    qc = query_to_cuda(q)
    if flags == rel.PLAN_SKETCH:
        plan = rel.plan_groupby(qc, flags=flags, groups_hint=len(np.unique(q["cols"][0])))
    else:
        plan = rel.plan_groupby(qc, flags=flags)
    k, a = rel.groupby(qc, plan=plan)
    torch.cuda.synchronize()
    gk, ga = canon_groupby(k, a)
    ek, ea = oracle.groupby(q)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(ga, ea)


def test_pinned_keys_are_the_heavy_hitters():
    q = CASES["four"]
    plan = rel.plan_groupby(query_to_cuda(q), flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    assert plan.n_hot == 4 and plan.tiny_slots == 4  # the fewest collision-free slots
    assert sorted(plan.hot_keys[:4]) == sorted(synth.mix64_signed(i) for i in (1, 2, 3, 4))
    qz = CASES["zipf"]
    plan = rel.plan_groupby(query_to_cuda(qz), flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    assert plan.n_hot >= 1 and plan.hot_keys[0] == synth.mix64_signed(1)
    assert plan.smem_slots > 0  # warm keys still have a CTA-shared layer


def test_bad_hot_keys_rejected():
    q = CASES["four"]
    qc = query_to_cuda(q)
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    plan.n_hot = 2
    plan.hot_keys[1] = plan.hot_keys[0]  # two keys on one slot
    with pytest.raises(rel.RelError) as e:
        rel.groupby(qc, plan=plan)
    assert e.value.status == rel.REL_E_INVALID


def test_sketch_batched_matches_oracle():
    names = list(CASES)
    qs = [query_to_cuda(CASES[n]) for n in names]
    infos = rel.sketch_batched(qs)
    for n, s in zip(names, infos):
        e = oracle.sketch(CASES[n])
        for f in ("sample_rows", "kept", "ndv", "singletons", "runs", "key_min", "key_max",
                  "key_bits"):
            assert getattr(s, f) == e[f], (n, f)
        assert list(s.top_key) == e["top_key"].tolist()
        assert list(s.top_count) == e["top_count"].tolist()
        assert bytes(s.hll) == e["hll"].tobytes()
        single = rel.sketch(query_to_cuda(CASES[n]))
        assert bytes(single.features) == bytes(s.features)


@pytest.mark.parametrize("key_type", ["int64", "int32"])
@pytest.mark.parametrize("n,offset", [(1, 0), (4097, 1), (1_000_003, 0), (3_000_001, 3)])
def test_key_hll_registers_match_oracle(key_type, n, offset):
    """The full-data HyperLogLog: registers bit for bit as the oracle's, over
    ragged sizes and unaligned columns (scalar loads)."""
    dt = np.int64 if key_type == "int64" else np.int32
    lo, hi = (-(2**62), 2**62) if key_type == "int64" else (-(2**31), 2**31 - 1)
    k = synth.uniform(n + offset, lo, hi, seed=n, tag=7, dtype=dt)
    regs, est = rel.key_hll(cuda(k)[offset:])
    eregs, eest = oracle.key_hll(k[offset:])
    np.testing.assert_array_equal(regs, eregs)
    assert abs(est - eest) <= 1e-9 * max(1.0, eest)


def test_learned_plan_sizes_long_tails_by_hyperloglog():
    """A large input whose sample saw its keys once: the learned plan sizes
    from the full-data HyperLogLog (within its error, 25 % headroom) instead
    of the network's guess, and the group-by is exact."""
    from paper_2608_13696_gb300 import planner

    if not os.path.exists(planner.DEFAULT_WEIGHTS):
        pytest.skip("no trained network")
    planner.use_default()
    # 6e6 rows over 3e6 key values: ~2.6e6 groups, a sample of singletons
    k = synth.uniform(6_000_000, 0, 3_000_000, seed=71, tag=1)
    v = synth.uniform(6_000_000, -9, 9, seed=71, tag=2)
    qc = {"cols": [cuda(k), cuda(v)], "keys": [0], "preds": [],
          "aggs": [("sum", 1, []), ("count", 1, [])]}
    plan = rel.plan_groupby(qc, flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH)
    true = np.unique(k).size
    assert plan.flags & rel.PLAN_HLL_SIZED
    lo, hi = 1.25 * true * (1 - 0.05), 1.25 * true * (1 + 0.05) + 1
    assert min(lo, len(k)) <= plan.est_groups <= min(hi, len(k))  # never above the rows
    keys, aggs, p2 = rel.groupby_auto(qc, flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH)
    assert not (p2.flags & rel.PLAN_FELL_BACK)
    ek, ea = oracle.groupby(oracle.kv_query(k, v, ops=("sum", "count")))
    gk, ga = canon_groupby(keys, aggs)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(ga, ea)
