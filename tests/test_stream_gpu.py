"""GPU parity of the streaming key/value group-by kernel (gb_stream): every
layer combination (pinned keys, shared table, global table), int32 and int64
keys, 4 and 2 aggregates, ragged tails, unaligned columns (scalar loads) and
the INT64_MIN side path, bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, cuda

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min


def inputs():
    zk, zv = synth.zipf_kv(700_003, seed=31, n_ranks=50_000)
    zk[::9973] = I64_MIN
    k32 = synth.uniform(300_001, -3000, 3000, seed=32, tag=3, dtype=np.int32)
    v32 = synth.uniform(300_001, -10**6, 10**6, seed=32, tag=4)
    fk, fv = synth.few_keys_kv(500_001, n_keys=5, seed=33)
    return {"zipf64": (zk, zv), "uni32": (k32, v32), "five64": (fk, fv)}


IN = inputs()
OPS = {4: ("sum", "count", "min", "max"), 2: ("sum", "count")}


def run(name, na, flags, layers=None, offset=0):
    k, v = IN[name]
    q = oracle.kv_query(k[offset:], v[offset:], ops=OPS[na])
    kc = cuda(k)[offset:]
    vc = cuda(v)[offset:]
    qc = {"cols": [kc, vc], "keys": [0], "preds": [], "aggs": [(o, 1, []) for o in OPS[na]]}
    plan = rel.plan_groupby(qc, flags=flags)
    if layers:
        plan.layers(*layers)
    rel.profile_start()
    keys, aggs = rel.groupby(qc, plan=plan)
    names = [n for n, _ in rel.profile_stop()]
    ek, ea = oracle.groupby(q)
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, ek)
    assert np.array_equal(ga, ea)
    return names, plan


@pytest.mark.parametrize("na", [4, 2])
@pytest.mark.parametrize("name", list(IN))
@pytest.mark.parametrize("offset", [0, 1])
def test_global_only(name, na, offset):
    names, _ = run(name, na, rel.PLAN_EXACT, layers=(0, 0, rel.VAR_GLOBAL), offset=offset)
    assert "gb_stream" in names


@pytest.mark.parametrize("na", [4, 2])
@pytest.mark.parametrize("name", list(IN))
def test_shared_table(name, na):
    names, _ = run(name, na, rel.PLAN_EXACT, layers=(0, 512, rel.VAR_SMEM))
    assert "gb_stream" in names


@pytest.mark.parametrize("na", [4, 2])
@pytest.mark.parametrize("name", ["zipf64", "five64"])
@pytest.mark.parametrize("offset", [0, 3])
def test_pinned(name, na, offset):
    names, plan = run(name, na, rel.PLAN_EXACT | rel.PLAN_SKETCH |
                      rel.plan_force(rel.VAR_GLOBAL), offset=offset)
    assert plan.n_hot > 0
    assert "gb_stream" in names


def test_pinned_with_shared_table():
    k, v = IN["zipf64"]
    qc = {"cols": [cuda(k), cuda(v)], "keys": [0], "preds": [],
          "aggs": [(o, 1, []) for o in OPS[4]]}
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH |
                            rel.plan_force(rel.VAR_SMEM))
    plan.smem_slots = 512  # small enough for the streaming kernel; pins kept
    assert plan.n_hot > 0
    rel.profile_start()
    keys, aggs = rel.groupby(qc, plan=plan)
    names = [n for n, _ in rel.profile_stop()]
    ek, ea = oracle.groupby(oracle.kv_query(k, v))
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, ek) and np.array_equal(ga, ea)
    assert "gb_stream" in names


def test_overflow_reported():
    k, v = IN["uni32"]
    qc = {"cols": [cuda(k), cuda(v)], "keys": [0], "preds": [],
          "aggs": [(o, 1, []) for o in OPS[2]]}
    plan = rel.plan_groupby(qc, flags=0, groups_hint=100).layers(0, 0, rel.VAR_GLOBAL)
    plan.slots = 256  # 6001 groups cannot fit
    with pytest.raises(rel.RelError) as e:
        rel.groupby(qc, plan=plan)
    assert e.value.status == rel.REL_E_OVERFLOW


@pytest.mark.parametrize("name", list(IN))
@pytest.mark.parametrize("offset", [0, 1])
def test_exact_count_streaming(name, offset):
    # the exact pre-pass of a one-key, unfiltered input runs the streaming
    # key-set kernel; its count is the number of distinct keys (INT64_MIN
    # counted once)
    k, v = IN[name]
    kc = cuda(k)[offset:]
    qc = {"cols": [kc, cuda(v)[offset:]], "keys": [0], "preds": [],
          "aggs": [("sum", 1, [])]}
    rel.profile_start()
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT)
    names = [n for n, _ in rel.profile_stop()]
    assert names == ["gb_main_keyset"]
    assert plan.est_groups == len(np.unique(k[offset:]))
    for n in (0, 1, 1023, 1025):
        qs = {"cols": [kc[:n], cuda(v)[offset:offset + n]], "keys": [0], "preds": [],
              "aggs": [("sum", 1, [])]}
        assert rel.plan_groupby(qs, flags=rel.PLAN_EXACT).est_groups == len(np.unique(k[offset:offset + n]))


@pytest.mark.parametrize("variant", [rel.VAR_GLOBAL, rel.VAR_SMEM, rel.VAR_PARTITIONED])
@pytest.mark.parametrize("name", ["zipf64", "uni32"])
def test_staged_path_still_exact(name, variant):
    # a plan that fixes the staging tile keeps the TMA-staged kernels (the
    # streaming ones take no tile size): both paths must agree with the oracle
    k, v = IN[name]
    qc = {"cols": [cuda(k), cuda(v)], "keys": [0], "preds": [],
          "aggs": [(o, 1, []) for o in OPS[4]]}
    plan = rel.plan_groupby(qc, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH | rel.plan_force(variant))
    plan.tile_rows, plan.n_stages = 1024, 3
    rel.profile_start()
    keys, aggs = rel.groupby(qc, plan=plan)
    names = [n for n, _ in rel.profile_stop()]
    assert "gb_stream" not in names
    ek, ea = oracle.groupby(oracle.kv_query(k, v))
    gk, ga = canon_groupby(keys, aggs)
    assert np.array_equal(gk, ek) and np.array_equal(ga, ea)


@pytest.mark.parametrize("name", list(IN))
@pytest.mark.parametrize("na", [4, 2])
def test_partitioned_streaming_passes(name, na):
    k, v = IN[name]
    q = oracle.kv_query(k, v, ops=OPS[na])
    qc = {"cols": [cuda(k), cuda(v)], "keys": [0], "preds": [],
          "aggs": [(o, 1, []) for o in OPS[na]]}
    for flags in (rel.PLAN_EXACT, rel.PLAN_EXACT | rel.PLAN_SKETCH):
        plan = rel.plan_groupby(qc, flags=flags | rel.plan_force(rel.VAR_PARTITIONED))
        rel.profile_start()
        keys, aggs = rel.groupby(qc, plan=plan)
        names = [n for n, _ in rel.profile_stop()]
        assert names[:2] == ["gb_part_hist", "gb_part_scan"]
        ek, ea = oracle.groupby(q)
        gk, ga = canon_groupby(keys, aggs)
        assert np.array_equal(gk, ek) and np.array_equal(ga, ea)
