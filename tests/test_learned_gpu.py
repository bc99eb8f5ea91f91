"""The learned sizing step (REL_PLAN_LEARNED) and the one-call group-by with
its overflow fallback (rel_groupby_auto): whatever the network predicts, the
result must equal the oracle group-by bit for bit; forced variants likewise.
The estimate and variant rules are checked with networks built by hand."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp as M
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, query_to_cuda

pytestmark = pytest.mark.gpu


def cases():
    li = synth.lineitem(200_000, seed=13)
    zk, zv = synth.zipf_kv(600_000, seed=14, n_ranks=200_000)
    fk, fv = synth.few_keys_kv(300_000, n_keys=4, seed=15)
    uk = synth.uniform_mixed(400_000, 1, 300_000, seed=16, tag=synth.TAG_KEY)
    uv = synth.uniform(400_000, -10**6, 10**6, seed=16, tag=synth.TAG_VAL)
    k32 = synth.uniform(70_000, -1000, 1000, seed=17, tag=3, dtype=np.int32)
    sent = np.array([np.iinfo(np.int64).min] * 10 + list(range(90)), dtype=np.int64)
    return {
        "lineitem": oracle.lineitem_query(li),
        "zipf": oracle.kv_query(zk, zv),
        "four": oracle.kv_query(fk, fv),
        "uniform_many": oracle.kv_query(uk, uv),
        "int32": oracle.kv_query(k32, zv[:70_000]),
        "sentinel": oracle.kv_query(sent, sent),
        "empty": oracle.kv_query(zk[:0], zv[:0]),
        "filtered_out": oracle.lineitem_query(synth.lineitem(9000, seed=18), date_hi=-1),
    }


CASES = cases()


def net(b3, seed=None):
    """Zero weights and the given output biases, or random weights."""
    p = np.zeros(M.N_PARAMS, np.float32) if seed is None else synth.mlp_params(seed)
    if b3 is not None:
        p[M.OFF_B3:] = b3
    return torch.from_numpy(p).cuda()


def check(q, keys, aggs):
    ek, ea = oracle.groupby(q)
    k, a = canon_groupby(keys, aggs)
    assert np.array_equal(k, ek)
    assert np.array_equal(a, ea)


def test_learned_needs_a_network():
    rel.planner_set(None)
    with pytest.raises(rel.RelError):
        rel.groupby_auto(query_to_cuda(CASES["zipf"]), flags=rel.PLAN_LEARNED)


@pytest.mark.parametrize("flags", [rel.PLAN_LEARNED, rel.PLAN_LEARNED | rel.PLAN_SKETCH])
@pytest.mark.parametrize("name", list(CASES))
def test_learned_random_network_exact(name, flags):
    rel.planner_set(net(None, seed=50))
    q = CASES[name]
    keys, aggs, plan = rel.groupby_auto(query_to_cuda(q), flags=flags)
    check(q, keys, aggs)


def test_underestimate_falls_back_to_exact():
    # y0 = 0: the estimate is the sample's distinct keys (<= 4096), far below
    # the 300k groups, so the first run overflows and the call re-plans
    rel.planner_set(net([0.0, 5.0, 0.0, 0.0]))
    q = CASES["uniform_many"]
    keys, aggs, plan = rel.groupby_auto(query_to_cuda(q), flags=rel.PLAN_LEARNED)
    check(q, keys, aggs)
    assert plan.flags & rel.PLAN_FELL_BACK
    assert plan.flags & rel.PLAN_EXACT
    assert plan.est_groups == len(oracle.groupby(q)[0])


def test_estimate_rule():
    # y0 = log2(1000): est = max(ceil(1.25 * 2 * 1000), sample distinct keys)
    rel.planner_set(net([np.log2(1000.0), 0.0, 0.0, 0.0]))
    for name, want in (("four", 2500), ("zipf", None)):
        qc = query_to_cuda(CASES[name])
        s = rel.sketch(qc)
        plan = rel.plan_groupby(qc, flags=rel.PLAN_LEARNED)
        assert plan.est_groups == max(2500, s.ndv)
        if want:
            assert plan.est_groups == want
    # never above the rows
    qc = query_to_cuda(CASES["sentinel"])
    assert rel.plan_groupby(qc, flags=rel.PLAN_LEARNED).est_groups == 100


@pytest.mark.parametrize("name,eligible", [("zipf", True), ("lineitem", False)])
def test_variant_rule(name, eligible):
    # the network prefers the partitioned variant; only key/value inputs may use it
    rel.planner_set(net([20.0, 0.0, 1.0, 9.0]))
    qc = query_to_cuda(CASES[name])
    plan = rel.plan_groupby(qc, flags=rel.PLAN_LEARNED)
    assert plan.variant == (rel.VAR_PARTITIONED if eligible else rel.VAR_GLOBAL)
    rel.planner_set(net([3.0, 9.0, 1.0, 0.0]))
    assert rel.plan_groupby(qc, flags=rel.PLAN_LEARNED).variant == rel.VAR_SMEM


@pytest.mark.parametrize("variant", [rel.VAR_SMEM, rel.VAR_GLOBAL, rel.VAR_PARTITIONED])
@pytest.mark.parametrize("name", ["zipf", "four", "uniform_many", "int32"])
def test_forced_variants_exact(name, variant):
    q = CASES[name]
    qc = query_to_cuda(q)
    for base in (rel.PLAN_EXACT, rel.PLAN_EXACT | rel.PLAN_SKETCH):
        keys, aggs, plan = rel.groupby_auto(qc, flags=base | rel.plan_force(variant))
        assert plan.variant == variant
        check(q, keys, aggs)


def test_forced_partitioned_rejected_for_filtered_input():
    with pytest.raises(rel.RelError) as e:
        rel.plan_groupby(query_to_cuda(CASES["lineitem"]),
                         flags=rel.PLAN_EXACT | rel.plan_force(rel.VAR_PARTITIONED))
    assert e.value.status == rel.REL_E_UNSUPPORTED


def test_auto_workspace_too_small():
    import ctypes

    L = rel.load()
    qc = query_to_cuda(CASES["zipf"])
    d = rel._Desc(qc)
    need = int(L.rel_groupby_auto_ws_bytes(ctypes.byref(d.d)))
    assert need == rel.auto_ws_bytes(qc)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty(16, dtype=torch.int64, device="cuda")
    ptrs = (ctypes.c_void_p * 4)(*([out.data_ptr()] * 4))
    n = ctypes.c_int64(-7)
    r = L.rel_groupby_auto(ctypes.byref(d.d), rel.PLAN_EXACT, ws.data_ptr(), need - 256,
                           out.data_ptr(), ptrs, 16, ctypes.byref(n), None, None)
    assert r == rel.REL_E_CAPACITY and n.value == -7


def test_forced_partitioned_many_groups():
    # ~24M distinct keys: the partition tables cannot hold them all, so the
    # spill table must take the rest without overflowing
    from synth import gpu as G

    n = 24_000_000
    k, v = G.kv(0, 0.0, n, 1 << 60, seed=21)
    qc = {"cols": [k, v], "keys": [0], "preds": [],
          "aggs": [("sum", 1, []), ("count", 1, []), ("min", 1, []), ("max", 1, [])]}
    keys, aggs, plan = rel.groupby_auto(qc, flags=rel.PLAN_EXACT |
                                        rel.plan_force(rel.VAR_PARTITIONED))
    assert plan.variant == rel.VAR_PARTITIONED
    kn = k.cpu().numpy()
    uk, cnt = np.unique(kn, return_counts=True)
    assert keys.numel() == uk.size
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, uk)
    assert np.array_equal(ga[1], cnt)
    assert int(ga[0].sum()) == int(v.sum().item())
