"""Full-size parity of the group-bys the benchmark times: 2e8 (int64 key,
int64 value) rows, keys Zipf(1.1) over 1e7 ranks (6.7e6 distinct) and 4
distinct keys; sum, count, min, max.  Every group the GPU produces is compared
with the oracle's, element by element and bit for bit (exact int64), for the
plain plan the benchmark uses (exact distinct count + sample sketch), the
learned plan (sketch + network, exact fallback) and forced variants.

The oracle is the plain CPU group-by; at this size it runs on hash partitions
of the rows, one thread per host core (oracle.partitioned, itself checked
against the single-threaded oracle), so each reference takes seconds."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import partitioned
from paper_2608_13696_gb300 import planner, rel

from gpu_util import canon_groupby, cuda

pytestmark = pytest.mark.gpu

N_BIG = 200_000_000


def _dataset(kind):
    if kind == "zipf":
        keys, vals = synth.zipf_kv(N_BIG, seed=0)
    else:
        keys, vals = synth.few_keys_kv(N_BIG, n_keys=4, seed=0)
    ek, ea = partitioned.groupby(oracle.kv_query(keys, vals), sort=True)
    return keys, vals, ek, ea


@pytest.fixture(scope="module", params=["zipf", "fourkeys"])
def big(request):
    keys, vals, ek, ea = _dataset(request.param)
    q = {"cols": [cuda(keys), cuda(vals)], "keys": [0], "preds": [],
         "aggs": [("sum", 1, []), ("count", 1, []), ("min", 1, []), ("max", 1, [])]}
    yield request.param, q, ek, ea
    del q
    torch.cuda.empty_cache()


def _assert_every_group(got, ek, ea):
    gk, ga = got
    assert gk.shape == ek.shape, (gk.shape, ek.shape)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(ga, ea)


def test_plain_plan_every_group(big):
    """The benchmark's plan: exact distinct count, then the sketch's pins."""
    kind, q, ek, ea = big
    plan = rel.plan_groupby(q, flags=rel.PLAN_EXACT | rel.PLAN_SKETCH)
    assert plan.est_groups == len(ek)
    if kind == "zipf":
        assert plan.variant == rel.VAR_PARTITIONED
    else:
        assert plan.n_hot == 4  # every key pinned in thread-private accumulators
    _assert_every_group(canon_groupby(*rel.groupby(q, plan=plan)), ek, ea)


@pytest.mark.parametrize("variant,sketch", [(rel.VAR_GLOBAL, True), (rel.VAR_PARTITIONED, False),
                                            (rel.VAR_SMEM, True)])
def test_forced_variants_every_group(big, variant, sketch):
    kind, q, ek, ea = big
    flags = rel.plan_force(variant) | (rel.PLAN_SKETCH if sketch else 0)
    plan = rel.plan_groupby(q, flags=flags, groups_hint=len(ek))
    _assert_every_group(canon_groupby(*rel.groupby(q, plan=plan)), ek, ea)


def test_learned_plan_every_group(big):
    """Learned sizing with the committed network; an overflowing estimate is
    re-planned exactly inside the call -- the result is exact either way."""
    import os

    if not os.path.exists(planner.DEFAULT_WEIGHTS):
        pytest.skip("no trained network")
    kind, q, ek, ea = big
    planner.use_default()
    keys, aggs, plan = rel.groupby_auto(q, flags=rel.PLAN_LEARNED | rel.PLAN_SKETCH)
    _assert_every_group(canon_groupby(keys, aggs), ek, ea)
    # the Zipf sample sees most keys once: the full-data HyperLogLog sizes the
    # plan and no exact re-plan is needed
    assert not (plan.flags & rel.PLAN_FELL_BACK), plan
    if kind == "zipf":
        assert plan.flags & rel.PLAN_HLL_SIZED
