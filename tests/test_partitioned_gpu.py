"""GPU parity of the partitioned group-by (REL_VAR_PARTITIONED: histogram,
scan, scatter into hash partitions, one shared-memory table per partition)
against the oracle, including pinned heavy hitters, partitions that overflow
their table (spilled to the global table), INT64_MIN keys and int32 keys."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, query_to_cuda

pytestmark = pytest.mark.gpu


def run(q, flags=rel.PLAN_EXACT, tweak=None):
    qc = query_to_cuda(q)
    plan = rel.plan_groupby(qc, flags=flags)
    if tweak:
        tweak(plan)
    assert plan.variant == rel.VAR_PARTITIONED, plan
    k, a = rel.groupby(qc, plan=plan)
    torch.cuda.synchronize()
    gk, ga = canon_groupby(k, a)
    ek, ea = oracle.groupby(q)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(ga, ea)
    return plan


@pytest.mark.parametrize("flags", [rel.PLAN_EXACT, rel.PLAN_EXACT | rel.PLAN_SKETCH])
def test_zipf(flags):
    keys, vals = synth.zipf_kv(600_001, seed=11, n_ranks=200_000)
    plan = run(oracle.kv_query(keys, vals), flags)
    if flags & rel.PLAN_SKETCH:
        assert plan.n_hot > 0  # the skewed head is pinned, not partitioned


def test_uniform_many_groups_sum_count():
    keys = synth.uniform_mixed(500_000, 1, 300_000, seed=12, tag=3)
    vals = synth.uniform(500_000, -10**6, 10**6, seed=12, tag=4)
    run(oracle.kv_query(keys, vals, ops=("count", "sum")))


def test_int32_keys_and_extremes():
    k = synth.uniform(400_000, -(2**31), 2**31 - 1, seed=13, tag=5, dtype=np.int32)
    k[::3] = k[7]
    v = synth.uniform(400_000, -(2**63), 2**63 - 1, seed=13, tag=6)
    run(oracle.kv_query(k, v, ops=("max", "min", "count", "sum")))


def test_sentinel_key_goes_to_side_path():
    keys, vals = synth.zipf_kv(300_000, seed=14, n_ranks=100_000)
    keys[::97] = np.iinfo(np.int64).min
    run(oracle.kv_query(keys, vals), rel.PLAN_EXACT | rel.PLAN_SKETCH)


def test_overflowing_partition_tables_spill():
    keys, vals = synth.zipf_kv(200_000, seed=15, n_ranks=60_000)

    def tiny_tables(plan):
        plan.part_bits = 4     # 16 partitions of ~2500 keys ...
        plan.smem_slots = 256  # ... into 256-slot tables: every partition spills

    run(oracle.kv_query(keys, vals), rel.PLAN_EXACT, tiny_tables)


def test_many_partitions_few_rows():
    keys, vals = synth.zipf_kv(5_000, seed=16, n_ranks=4_000)

    def many(plan):  # ~1000 groups: the planner would not partition; force it
        plan.variant, plan.part_bits, plan.smem_slots = rel.VAR_PARTITIONED, 12, 256
        plan.tiny_slots, plan.n_hot = 0, 0
        plan.slots = 1 << 16

    run(oracle.kv_query(keys, vals), rel.PLAN_EXACT, many)


def test_bad_partition_plan_rejected():
    keys, vals = synth.zipf_kv(50_000, seed=17, n_ranks=20_000)
    qc = query_to_cuda(oracle.kv_query(keys, vals))
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT)
    plan.part_bits = 15  # above the 16384-partition limit
    with pytest.raises(rel.RelError) as e:
        rel.groupby(qc, plan=plan)
    assert e.value.status == rel.REL_E_INVALID


@pytest.mark.parametrize("bits", [8, 9, 11, 14])
def test_two_level_scatter(bits):
    # above 2^8 partitions the scatter runs in two levels (bins of
    # 2^(bits-8) partitions, then partitions); skewed keys make bins of many
    # tiles next to empty ones
    keys, vals = synth.zipf_kv(1_000_003, seed=18 + bits, n_ranks=400_000)
    keys[::113] = np.iinfo(np.int64).min

    def force(plan):
        plan.part_bits = bits
        plan.smem_slots = max(256, min(4096, 1 << (20 - bits)))

    run(oracle.kv_query(keys, vals), rel.PLAN_EXACT | rel.PLAN_SKETCH, force)


@pytest.mark.parametrize("ops,key_dtype", [(("sum", "count"), np.int64), (("count", "sum"), np.int32),
                                           (("max", "min", "count", "sum"), np.int32)])
def test_two_level_scatter_pinned_shapes(ops, key_dtype):
    # pinned heavy hitters with both aggregate widths and both key types,
    # through the two scatter levels (2^10 partitions)
    keys, vals = synth.zipf_kv(700_001, seed=31, n_ranks=250_000)
    keys = keys.astype(key_dtype)

    def force(plan):
        plan.part_bits = 10
        plan.smem_slots = 1024

    plan = run(oracle.kv_query(keys, vals, ops=ops), rel.PLAN_EXACT | rel.PLAN_SKETCH, force)
    assert plan.n_hot > 0
