"""The C-ABI library: it loads, it exports exactly what include/rel.h declares,
and host-side validation and sizing work without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2608_13696_gb300 import build as B
from paper_2608_13696_gb300 import rel

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "rel.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rel_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return rel.load()


def test_header_matches_binding_list():
    assert declared_functions() == sorted(rel.EXPORTS)


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_version_and_counters(L):
    assert L.rel_version() == 100
    assert L.rel_launch_count() == 0  # nothing launched in this process
    assert L.rel_last_error() is not None


def test_ws_sizes(L):
    assert L.rel_groupby_ws_bytes(16, 4) == 256 + 16 * 8 * 5
    assert L.rel_groupby_ws_bytes(1 << 20, 2) == 256 + (1 << 20) * 24
    # join: next_pow2(2n) slots x 16 B (key, build index) + the payload copy (n x 8 B,
    # rounded up to 256 B) + n x 16 B side list
    assert L.rel_join_ws_bytes(1_000_000) == 256 + (1 << 21) * 16 + 8_000_000 + 1_000_000 * 16
    assert L.rel_join_ws_bytes(0) == 256 + 16 * 16 + 256 + 16


def _desc(n_rows=100, **over):
    cols = (rel.Col * 2)(rel.Col(0x1000, rel.I64, 0), rel.Col(0x2000, rel.I64, 0))
    keys = (ctypes.c_int32 * 1)(0)
    aggs = (rel.Agg * 1)(rel.Agg(rel.OPS["sum"], 1, 0, 0))
    preds = (rel.RangePred * 1)()
    d = rel.GroupByDesc(n_rows, 2, 1, 0, 1, cols, keys, preds, aggs)
    for k, v in over.items():
        setattr(d, k, v)
    return d, (cols, keys, aggs, preds)


def test_plan_from_hint_is_host_only(L):
    d, keep = _desc()
    plan = rel.Plan()
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 1000, None, 0,
                           ctypes.byref(plan), None) == rel.REL_OK
    assert plan.est_groups == 1000 and plan.slots == 2048
    assert plan.variant == rel.VAR_SMEM and plan.smem_slots == 2048 and plan.tiny_slots == 8
    assert plan.workspace_bytes == L.rel_groupby_ws_bytes(2048, 1)
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 5, None, 0,
                           ctypes.byref(plan), None) == rel.REL_OK
    assert plan.tiny_slots == 8 and plan.smem_slots == 0  # thread-private accumulators only
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 10**7, None, 0,
                           ctypes.byref(plan), None) == rel.REL_OK
    assert plan.variant == rel.VAR_GLOBAL and plan.slots == 1 << 25
    assert plan.tiny_slots == 8 and plan.smem_slots == 2048  # caches in front of the table


def test_exact_plan_reports_scratch_without_gpu(L):
    d, keep = _desc(n_rows=1000)
    plan = rel.Plan()
    r = L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), rel.PLAN_EXACT, 0, None, 0,
                        ctypes.byref(plan), None)
    assert r == rel.REL_E_CAPACITY
    assert plan.scratch_bytes == 256 + 2048 * 8


@pytest.mark.parametrize("field,value", [
    ("n_rows", -1), ("n_cols", 0), ("n_cols", 9), ("n_keys", 0), ("n_keys", 5),
    ("n_aggs", 0), ("n_aggs", 9), ("n_preds", 5),
])
def test_invalid_descriptors_rejected_before_cuda(L, field, value):
    d, keep = _desc(**{field: value})
    plan = rel.Plan()
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 10, None, 0,
                           ctypes.byref(plan), None) == rel.REL_E_INVALID
    assert L.rel_last_error()


def test_bad_agg_and_packed_key_rejected(L):
    d, keep = _desc()
    keep[2][0].op = 7
    plan = rel.Plan()
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 10, None, 0,
                           ctypes.byref(plan), None) == rel.REL_E_INVALID
    # two int64 key columns cannot be packed into one 64-bit key
    d, keep = _desc()
    keys = (ctypes.c_int32 * 2)(0, 1)
    d.keys_ref = keys
    d.key_cols = keys
    d.n_keys = 2
    assert L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), 0, 10, None, 0,
                           ctypes.byref(plan), None) == rel.REL_E_INVALID


def test_groupby_agg_argument_checks(L):
    d, keep = _desc()
    plan = rel.Plan()
    plan.slots = 24  # not a power of two
    n = ctypes.c_int64()
    assert L.rel_groupby_agg(ctypes.byref(d), ctypes.byref(plan), 0x100, 1 << 20, 0x10, None, 0,
                             ctypes.byref(n), None) == rel.REL_E_INVALID
    plan.slots = 1024
    plan.smem_slots = 24
    assert L.rel_groupby_agg(ctypes.byref(d), ctypes.byref(plan), 0x100, 1 << 20, 0x10, None, 0,
                             ctypes.byref(n), None) == rel.REL_E_INVALID
    plan.smem_slots = 0
    plan.tiny_slots = 12
    assert L.rel_groupby_agg(ctypes.byref(d), ctypes.byref(plan), 0x100, 1 << 20, 0x10, None, 0,
                             ctypes.byref(n), None) == rel.REL_E_INVALID
    plan.tiny_slots = 0
    # workspace too small: capacity error before any device work
    assert L.rel_groupby_agg(ctypes.byref(d), ctypes.byref(plan), 0x100, 100, 0x10, None, 0,
                             ctypes.byref(n), None) == rel.REL_E_CAPACITY
    # a workspace off a 256-byte boundary is rejected before any device work
    assert L.rel_groupby_agg(ctypes.byref(d), ctypes.byref(plan), 0x110, 1 << 20, 0x10, None, 0,
                             ctypes.byref(n), None) == rel.REL_E_INVALID
    assert b"aligned" in L.rel_last_error()


def test_static_groupby_checks_before_any_device_work(L):
    d, keep = _desc()
    n = ctypes.c_int64()
    out = (ctypes.c_void_p * 1)(0x3000)
    # max_groups outside 1..REL_STATIC_MAX_GROUPS
    for bad in (0, rel.STATIC_MAX_GROUPS + 1):
        assert L.rel_groupby_agg_static(ctypes.byref(d), bad, 0x3000, out, 10, ctypes.byref(n),
                                        None) == rel.REL_E_UNSUPPORTED
        assert b"max_groups" in L.rel_last_error()
    # the host count carries the overflow check: NULL is refused
    assert L.rel_groupby_agg_static(ctypes.byref(d), 16, 0x3000, out, 10, None,
                                    None) == rel.REL_E_INVALID
    assert b"n_groups_host" in L.rel_last_error()


def test_learned_rule_on_synthetic_network_outputs(L):
    """The learned sizing rule, host only: est = min(rows, ceil(1.25 * 2^(clamp(y0, 0, 61)
    + 1))), never below the sample's distinct keys; variant = largest allowed logit."""
    info = rel.SketchInfo()
    info.ndv = 7
    nan = float("nan")
    cases = [  # (y, rows, partitioned_ok) -> (est, variant)
        ((10.0, 1.0, 3.0, 2.0), 10**6, True, (2560, rel.VAR_GLOBAL)),
        ((10.0, 1.0, 3.0, 4.0), 10**6, True, (2560, rel.VAR_PARTITIONED)),
        ((10.0, 1.0, 3.0, 4.0), 10**6, False, (2560, rel.VAR_GLOBAL)),
        ((10.0, 2.0, 2.0, 2.0), 10**6, True, (2560, rel.VAR_SMEM)),
        ((-5.0, 0.0, 0.0, 0.0), 10**6, True, (7, rel.VAR_SMEM)),  # ceil(2.5) = 3 < ndv
        ((0.5, 0.0, 0.0, 0.0), 10**6, True, (7, rel.VAR_SMEM)),   # ceil(1.25 * 2^1.5) = 4 -> ndv
        ((3.0, 0.0, 0.0, 0.0), 10**6, True, (20, rel.VAR_SMEM)),  # 1.25 * 16
        ((40.0, 0.0, 1.0, 0.0), 1000, True, (1000, rel.VAR_GLOBAL)),
        ((nan, 0.0, 1.0, 0.0), 12345, True, (12345, rel.VAR_GLOBAL)),
        ((100.0, 0.0, 0.0, 0.0), 1 << 62, True, (1 << 62, rel.VAR_SMEM)),  # clamp at 61: 1.25*2^62
    ]
    for y, rows, pok, want in cases:
        got = rel.plan_learned_rule(info, y, rows, pok)
        assert got == want, (y, rows, pok, got, want)
    est, var = ctypes.c_int64(), ctypes.c_int32()
    assert L.rel_plan_learned_rule(None, None, 10, 1, ctypes.byref(est),
                                   ctypes.byref(var)) == rel.REL_E_INVALID


def test_batched_plan_checks_before_any_device_work(L):
    d, keep = _desc()
    plans = (rel.Plan * 1)()
    n1 = L.rel_plan_size_batched_ws_bytes(1)
    assert L.rel_plan_size_batched_ws_bytes(100) > n1 >= L.rel_sketch_batched_ws_bytes(1)
    assert L.rel_plan_size_batched(ctypes.byref(d), 1, rel.PLAN_EXACT, None, 0, plans,
                                   None) == rel.REL_E_UNSUPPORTED
    assert L.rel_plan_size_batched(ctypes.byref(d), 0, rel.PLAN_LEARNED, None, 0, plans,
                                   None) == rel.REL_OK
    L.rel_planner_set(None, None)
    assert L.rel_plan_size_batched(ctypes.byref(d), 1, rel.PLAN_LEARNED, None, 0, plans,
                                   None) == rel.REL_E_INVALID
    assert b"network" in L.rel_last_error()


def test_join_argument_checks(L):
    t = rel.JoinTableC()
    assert L.rel_join_build(None, None, -1, None, 0, ctypes.byref(t), None) == rel.REL_E_UNSUPPORTED
    assert L.rel_join_build(None, None, 1 << 31, None, 0, ctypes.byref(t), None) == rel.REL_E_UNSUPPORTED
    assert L.rel_join_build(None, None, 10, None, 0, ctypes.byref(t), None) == rel.REL_E_INVALID
    assert L.rel_join_build(0x10, 0x10, 10, 0x100, 10, ctypes.byref(t), None) == rel.REL_E_CAPACITY
    assert L.rel_join_build(0x10, 0x10, 10, 0x108, 1 << 20, ctypes.byref(t), None) == rel.REL_E_INVALID
    n = ctypes.c_int64()
    # an unbuilt handle is rejected
    assert L.rel_join_probe(ctypes.byref(t), 0x10, 10, 0x10, 0x10, 0x10, 10, ctypes.byref(n),
                            None) == rel.REL_E_INVALID


def test_planner_and_mlp_sizes_and_checks(L):
    # backward scratch: dz1, dz2, dout per sample (132 floats)
    assert L.rel_mlp_ws_bytes(256) == 256 * 132 * 4
    assert L.rel_mlp_ws_bytes(0) == 132 * 4
    assert L.rel_mlp_ws_bytes(-1) == 0
    # AdamW rejects a step < 1 and betas outside [0, 1) before any launch
    p = ctypes.c_void_p(0x1000)
    assert L.rel_mlp_adamw(p, p, p, p, p, 0, 1e-3, 0.9, 0.999, 1e-8, 0.0, None) == rel.REL_E_INVALID
    assert L.rel_mlp_adamw(p, p, p, p, p, 1, 1e-3, 1.0, 0.999, 1e-8, 0.0, None) == rel.REL_E_INVALID
    assert L.rel_mlp_forward(None, None, None, -1, None, None, None) == rel.REL_E_INVALID
    # the planner takes both parameter copies or neither
    assert L.rel_planner_set(p, None) == rel.REL_E_INVALID
    assert L.rel_planner_set(None, None) == rel.REL_OK


def test_learned_plan_needs_a_network_and_scratch(L):
    d, keep = _desc(100)
    plan = rel.Plan()
    assert L.rel_planner_set(None, None) == rel.REL_OK
    # without workspace: the scratch size comes back (sketch + 2 KB of features and
    # outputs + 16 KB of HyperLogLog registers) before any GPU work
    r = L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d), rel.PLAN_LEARNED, 0, None, 0,
                        ctypes.byref(plan), None)
    assert r == rel.REL_E_CAPACITY
    assert plan.scratch_bytes == L.rel_sketch_ws_bytes() + 2048 + 4 * 4096


def test_forced_partitioned_needs_key_value_shape(L):
    cols = (rel.Col * 3)(rel.Col(0x1000, rel.I64, 0), rel.Col(0x2000, rel.I64, 0),
                         rel.Col(0x3000, rel.I32, 0))
    keys = (ctypes.c_int32 * 1)(0)
    aggs = (rel.Agg * 1)(rel.Agg(rel.OPS["sum"], 1, 0, 0))
    preds = (rel.RangePred * 1)(rel.RangePred(2, 0, 0, 10))
    d = rel.GroupByDesc(100, 3, 1, 1, 1, cols, keys, preds, aggs)  # a filter: not key/value
    plan = rel.Plan()
    r = L.rel_plan_size(rel.OP_GROUPBY, ctypes.byref(d),
                        rel.plan_force(rel.VAR_PARTITIONED), 10, None, 0, ctypes.byref(plan), None)
    assert r == rel.REL_E_UNSUPPORTED


def test_auto_workspace_bound(L):
    d, keep = _desc(1_000_000)
    need = L.rel_groupby_auto_ws_bytes(ctypes.byref(d))
    # at least the layered table for 2n slots and the partition records
    assert need >= 256 + (1 << 21) * 16
    assert need >= 16 * 1_000_000
    bad, keep2 = _desc(-1)
    assert L.rel_groupby_auto_ws_bytes(ctypes.byref(bad)) == 0


def _batch_arrays(n_rows=1000, slots=2048, cap=100, key_type=None):
    g = (rel.BatchGroupBy * 1)()
    g[0].keys, g[0].vals, g[0].n_rows = 0x1000, 0x2000, n_rows
    g[0].key_type = rel.I64 if key_type is None else key_type
    g[0].n_aggs = 2
    g[0].ops[0], g[0].ops[1] = rel.OPS["sum"], rel.OPS["count"]
    g[0].slots, g[0].est_groups = slots, 10
    g[0].out_keys, g[0].out_capacity = 0x3000, cap
    g[0].out_aggs[0], g[0].out_aggs[1] = 0x4000, 0x5000
    j = (rel.BatchJoinC * 1)()
    j[0].build_keys, j[0].build_payload, j[0].n_build = 0x6000, 0x7000, 500
    j[0].probe_keys, j[0].n_probe = 0x8000, 4000
    j[0].out_probe_idx, j[0].out_build_idx, j[0].out_payload = 0x9000, 0xa000, 0xb000
    j[0].out_capacity = 4000
    return g, j


def test_batch_sizes_and_validation(L):
    g, j = _batch_arrays()
    need = L.rel_batch_ws_bytes(g, 1, j, 1)
    # tables: 2048 slots x (8 + 2 x 8) B, 1024 join slots x 24 B, side list 500 x 16 B
    assert need >= 2048 * 24 + 1024 * 24 + 500 * 16
    assert L.rel_batch_ws_bytes(g, 0, j, 0) > 0
    bad, j2 = _batch_arrays(slots=1000)          # not a power of two
    assert L.rel_batch_ws_bytes(bad, 1, j2, 1) == 0
    bad, j2 = _batch_arrays(key_type=rel.U8)     # u8 keys are not a key/value batch
    assert L.rel_batch_ws_bytes(bad, 1, j2, 1) == 0
    h = rel.BatchHandle()
    for cfg in ((100, 8, 1, 0), (256, 3, 1, 0), (256, 8, 3, 0), (256, 8, 1, 4096)):
        c = rel.BatchConfig(*cfg)
        r = L.rel_batch_prepare(g, 1, j, 1, ctypes.byref(c), ctypes.c_void_p(0x10000), need,
                                ctypes.byref(h), None)
        assert r == rel.REL_E_INVALID, cfg
    c = rel.BatchConfig(256, 8, 1, 0)
    r = L.rel_batch_prepare(g, 1, j, 1, ctypes.byref(c), ctypes.c_void_p(0x10000), need - 1,
                            ctypes.byref(h), None)
    assert r == rel.REL_E_CAPACITY
    # a handle that prepare never filled is refused
    assert L.rel_batch_run(ctypes.byref(rel.BatchHandle()), None) == rel.REL_E_INVALID


@pytest.mark.parametrize("ct", [rel.Col, rel.GroupByDesc, rel.BatchGroupBy, rel.BatchJoinC])
def test_numpy_layouts_match_ctypes(ct):
    # the batch and batched-sketch descriptors are filled column-wise in numpy
    # arrays that must have the C structs' exact layout
    dt = rel._np_dtype(ct)
    assert dt.itemsize == ctypes.sizeof(ct)
    for name, _ in ct._fields_:
        assert dt.fields[name][1] == getattr(ct, name).offset, name


def test_partitioned_workspace_holds_both_record_levels(L):
    # one 16-byte record per row, and above 2^8 partitions a second one per
    # row for the first scatter level (bins of partitions)
    n = 1_000_000
    sizes = {}
    for bits in (4, 8, 9, 14):
        plan = rel.Plan()
        plan.variant, plan.slots, plan.part_bits, plan.smem_slots = rel.VAR_PARTITIONED, 1 << 16, bits, 1024
        sizes[bits] = L.rel_plan_ws_bytes(ctypes.byref(plan), 4, n)
    assert 16 * n < sizes[4] <= sizes[8] < 16 * n + (1 << 26)
    assert sizes[9] - sizes[8] >= 16 * n
    assert sizes[14] - sizes[9] < (1 << 26)  # only per-partition arrays grow
    plan = rel.Plan()
    plan.variant, plan.slots, plan.part_bits = rel.VAR_PARTITIONED, 1 << 16, 15
    assert L.rel_plan_ws_bytes(ctypes.byref(plan), 4, n) == 0  # beyond 16384 partitions
