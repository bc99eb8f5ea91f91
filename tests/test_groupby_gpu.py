"""GPU parity of the fused filter + group-by against the oracle.

Every aggregate is exact int64, so the bar is bit-exact equality after
sorting by key.  Each case runs through the C ABI in every per-CTA table mode
(thread-private, CTA-shared, global) and with both the specialised and the
descriptor-interpreting kernel, at sizes spanning several tiles plus a
ragged tail (the full-size cases, every group compared, are in
test_fullsize_gpu.py)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, cuda, query_to_cuda
from test_oracle_groupby import rand_query

pytestmark = pytest.mark.gpu

# per-CTA layers: (thread-private slots, CTA-shared slots, variant label)
MODES = {"tiny": (8, 0, rel.VAR_SMEM), "shared": (0, 256, rel.VAR_SMEM),
         "global": (0, 0, rel.VAR_GLOBAL), "layered": (8, 1024, rel.VAR_GLOBAL)}


def gpu_groupby(q_np, mode=None, flags=0, hint=0, plan=None):
    qc = query_to_cuda(q_np)
    if plan is None:
        plan = rel.plan_groupby(qc, flags=flags, groups_hint=hint)
    if mode is not None:
        plan.layers(*MODES[mode])
    plan.flags |= flags & rel.PLAN_GENERIC
    k, a = rel.groupby(qc, plan=plan)
    torch.cuda.synchronize()
    return canon_groupby(k, a)


def assert_same(q_np, got):
    ek, ea = oracle.groupby(q_np)
    gk, ga = got
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(ga, ea)


@pytest.mark.parametrize("n", [0, 1, 17, 1000, 4097, 100_003])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("generic", [False, True])
def test_lineitem_shape(n, mode, generic):
    li = synth.lineitem(n, seed=n + 1)
    q = oracle.lineitem_query(li)
    assert_same(q, gpu_groupby(q, mode=mode, hint=8,
                               flags=rel.PLAN_GENERIC if generic else 0))


def test_lineitem_full_exact_plan():
    li = synth.lineitem(1_000_000, seed=0)
    q = oracle.lineitem_query(li)
    plan = rel.plan_groupby(query_to_cuda(q), flags=rel.PLAN_EXACT)
    assert plan.est_groups == 6 and plan.tiny_slots == 8 and plan.smem_slots == 0
    assert_same(q, gpu_groupby(q, plan=plan))


def test_lineitem_full_unsized_plan():
    """No hint, no exact pass: the table is sized for n_rows groups."""
    li = synth.lineitem(1_000_000, seed=0)
    q = oracle.lineitem_query(li)
    assert_same(q, gpu_groupby(q))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("generic", [False, True])
def test_zipf_kv(mode, generic):
    keys, vals = synth.zipf_kv(300_001, seed=2, n_ranks=50_000)
    q = oracle.kv_query(keys, vals)
    got = gpu_groupby(q, mode=mode, flags=rel.PLAN_EXACT | (rel.PLAN_GENERIC if generic else 0))
    assert_same(q, got)


def test_exact_plan_counts_distinct_keys():
    keys, vals = synth.zipf_kv(200_000, seed=3, n_ranks=30_000)
    q = oracle.kv_query(keys, vals)
    for generic in (0, rel.PLAN_GENERIC):
        plan = rel.plan_groupby(query_to_cuda(q), flags=rel.PLAN_EXACT | generic)
        assert plan.est_groups == len(np.unique(keys))


@pytest.mark.parametrize("mode", list(MODES))
def test_few_keys_and_int32_keys(mode):
    keys, vals = synth.few_keys_kv(123_457, n_keys=4, seed=4)
    q = oracle.kv_query(keys, vals)
    assert_same(q, gpu_groupby(q, mode=mode, hint=4))
    k32 = synth.uniform(123_457, -1000, 1000, seed=5, tag=9, dtype=np.int32)
    q32 = oracle.kv_query(k32, vals, ops=("max", "count", "sum"))
    assert_same(q32, gpu_groupby(q32, mode=mode, hint=2001))


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("mode", list(MODES))
def test_random_descriptors(seed, mode):
    rng = np.random.default_rng(1000 + seed)
    q = rand_query(rng, int(rng.integers(1, 9000)))
    assert_same(q, gpu_groupby(q, mode=mode, flags=rel.PLAN_EXACT))


@pytest.mark.parametrize("mode", list(MODES))
def test_sentinel_key_and_extremes(mode):
    rng = np.random.default_rng(9)
    k = rng.integers(-3, 3, 5000).astype(np.int64)
    k[::7] = np.iinfo(np.int64).min
    k[3::11] = np.iinfo(np.int64).max
    v = rng.integers(-(2**63), 2**63 - 1, 5000, dtype=np.int64)
    v[:4] = [np.iinfo(np.int64).min, np.iinfo(np.int64).max, 0, -1]
    q = oracle.kv_query(k, v)
    assert_same(q, gpu_groupby(q, mode=mode, hint=16))


@pytest.mark.parametrize("mode", list(MODES))
def test_all_rows_filtered_and_empty(mode):
    li = synth.lineitem(5000, seed=6)
    q = oracle.lineitem_query(li, date_hi=-1)
    k, a = gpu_groupby(q, mode=mode, hint=8)
    assert k.size == 0 and a.shape == (5, 0)


@pytest.mark.parametrize("mode", list(MODES))
def test_all_distinct_keys(mode):
    k = np.random.default_rng(3).permutation(np.arange(-20_000, 20_000, dtype=np.int64))
    v = np.arange(len(k), dtype=np.int64)
    q = oracle.kv_query(k, v, ops=("sum", "count"))
    assert_same(q, gpu_groupby(q, mode=mode, hint=len(k)))


def test_misaligned_columns_take_the_unstaged_path():
    keys, vals = synth.zipf_kv(50_001, seed=7, n_ranks=5000)
    q = oracle.kv_query(keys[1:], vals[1:])
    qc = query_to_cuda(oracle.kv_query(keys, vals))
    qc["cols"] = [c[1:] for c in qc["cols"]]  # 8-byte aligned, not 16
    for mode in MODES:
        plan = rel.plan_groupby(qc, groups_hint=5000)
        plan.layers(*MODES[mode])
        k, a = rel.groupby(qc, plan=plan)
        gk, ga = canon_groupby(k, a)
        ek, ea = oracle.groupby(q)
        np.testing.assert_array_equal(gk, ek)
        np.testing.assert_array_equal(ga, ea)


def test_capacity_error_reports_required_groups():
    keys, vals = synth.zipf_kv(20_000, seed=8, n_ranks=3000)
    q = oracle.kv_query(keys, vals)
    qc = query_to_cuda(q)
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT)
    ng = plan.est_groups
    k, a = rel.groupby(qc, plan=plan, capacity=5)  # retries after REL_E_CAPACITY
    assert k.numel() == ng
    assert_same(q, canon_groupby(k, a))


def test_overflow_is_reported_not_hung():
    keys, vals = synth.zipf_kv(100_000, seed=9, n_ranks=20_000)
    qc = query_to_cuda(oracle.kv_query(keys, vals))
    plan = rel.plan_groupby(qc, groups_hint=8)  # 16 slots for ~9000 groups
    plan.layers(0, 0, rel.VAR_GLOBAL)
    with pytest.raises(rel.RelError) as e:
        rel.groupby(qc, plan=plan)
    assert e.value.status == rel.REL_E_OVERFLOW
    # the same workspace and stream keep working afterwards
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT)
    k, _ = rel.groupby(qc, plan=plan)
    assert k.numel() == len(np.unique(keys))


def test_device_wait_gives_up_and_the_stream_stays_usable():
    """Failure detection without a GPU fault: under the test hook the staged
    kernel's consumers never hand a stage back, so the producer's bounded
    wait and then the consumers' run out (20 ms) and the call returns
    REL_E_TIMEOUT; the next call on the same stream is exact."""
    import time

    li = synth.lineitem(1_000_000, seed=5)
    q = oracle.lineitem_query(li)
    qc = query_to_cuda(q)
    plan = rel.plan_groupby(qc, groups_hint=8)
    plan.tile_rows, plan.n_stages = 256, 2  # CTAs get more tiles than stages
    plan.flags |= rel.PLAN_TEST_STALL
    t0 = time.perf_counter()
    with pytest.raises(rel.RelError) as e:
        rel.groupby(qc, plan=plan)
    assert e.value.status == rel.REL_E_TIMEOUT
    assert time.perf_counter() - t0 < 1.5  # the short test limit, not the 2 s one
    plan.flags &= ~rel.PLAN_TEST_STALL
    assert_same(q, canon_groupby(*rel.groupby(qc, plan=plan)))
    assert_same(q, gpu_groupby(q, flags=rel.PLAN_EXACT))


# ------------------------------------------ the exact pre-pass's key sets


@pytest.mark.parametrize("key_type,generic", [("int64", False), ("int32", False), ("int64", True)])
def test_exact_count_beyond_the_l2_sized_set(key_type, generic):
    """2.4e7 rows of ~2.4e7 distinct keys: more than the exact pre-pass's
    first, L2-sized key set holds (2^24 slots), so it overflows and the count
    comes from the full-size set -- still the exact number of distinct keys."""
    from synth import gpu as G

    n = 24_000_000
    k, v = G.kv(0, 0.0, n, 10**15, seed=11)
    if key_type == "int32":
        k = k.to(torch.int32)
    q = {"cols": [k, v], "keys": [0], "preds": [], "aggs": [("count", 1, [])]}
    plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT | (rel.PLAN_GENERIC if generic else 0))
    distinct = np.unique(k.cpu().numpy()).size
    assert distinct > (1 << 24)
    assert plan.est_groups == distinct


def test_exact_count_within_the_l2_sized_set():
    """2.4e7 rows over 1e7 keys: the first key set holds them all."""
    from synth import gpu as G

    k, v = G.kv(1, 1.1, 24_000_000, 10**7, seed=12)
    q = {"cols": [k, v], "keys": [0], "preds": [], "aggs": [("count", 1, [])]}
    plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT)
    assert plan.est_groups == np.unique(k.cpu().numpy()).size


@pytest.mark.parametrize("key_type", ["int64", "int32"])
@pytest.mark.parametrize("offset", [0, 1, 3])
@pytest.mark.parametrize("n", [1, 7, 2047, 2048 * 9 + 5, 1_000_003])
def test_exact_count_streaming_shapes(key_type, offset, n):
    """The streaming distinct count over ragged sizes, unaligned columns
    (scalar loads) and the INT64_MIN side key: equal to np.unique."""
    dt = np.int64 if key_type == "int64" else np.int32
    k = synth.uniform(n + offset, -5 * n, 5 * n, seed=n, tag=5, dtype=dt)
    if key_type == "int64" and n > 10:
        k[::11] = np.iinfo(np.int64).min
        k[1::13] = np.iinfo(np.int64).max
    v = synth.uniform(n + offset, -9, 9, seed=n, tag=6)
    kc, vc = cuda(k)[offset:], cuda(v)[offset:]
    q = {"cols": [kc, vc], "keys": [0], "preds": [], "aggs": [("count", 1, [])]}
    plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT)
    assert plan.est_groups == np.unique(k[offset:]).size


def test_exact_count_empty_input():
    kc = torch.empty(0, dtype=torch.int64, device="cuda")
    q = {"cols": [kc, kc], "keys": [0], "preds": [], "aggs": [("count", 1, [])]}
    assert rel.plan_groupby(q, flags=rel.PLAN_EXACT).est_groups == 0
