"""The planner driver end to end at toy scale (collect runs, train with the
library's kernels, evaluate), instances of the planner workload's recipe
checked against the oracle group-by, and the committed trained network's
gain over the exact pre-pass."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2608_13696_gb300 import planner, rel
from synth import gpu as G

from gpu_util import canon_groupby

pytestmark = pytest.mark.gpu


def test_collect_train_evaluate(tmp_path):
    runs = tmp_path / "runs.npz"
    d = planner.collect(range(12), str(runs), reps=1, rows_lo=50_000, rows_hi=400_000,
                        log_every=0)
    assert d["features"].shape == (12, 264)
    assert np.all(d["label"] >= 0) and np.all(d["label"] < 3)
    assert np.all(d["times_ms"] > 0)
    # the exact group count agrees with the rows/domain bounds
    meta = d["meta"]
    assert np.all(2.0 ** d["log2_groups"] <= np.minimum(meta[:, 1], meta[:, 2]) + 0.5)
    w = tmp_path / "w.npz"
    ck = tmp_path / "ck.npz"
    info = planner.train([str(runs)], str(w), epochs=3, batch=4, val_frac=0.25, ckpt=str(ck))
    assert info["val_metrics"]["epoch"] == 3
    # resume from the checkpoint: nothing left to do, same parameters
    info2 = planner.train([str(runs)], str(tmp_path / "w2.npz"), epochs=3, batch=4,
                          val_frac=0.25, ckpt=str(ck))
    assert np.array_equal(np.load(w)["params"], np.load(tmp_path / "w2.npz")["params"])
    r = planner.evaluate(range(100, 104), str(w), rows_lo=50_000, rows_hi=400_000, log_every=0)
    assert r["instances"] == 4 and r["mismatches"] == 0


@pytest.mark.parametrize("seed", range(8))
def test_recipe_instances_match_oracle(seed):
    # the planner workload's recipe at <= 2M rows, every family
    inst = G.instance(5000 + seed, rows_lo=200_000, rows_hi=2_000_000)
    if seed < len(G.FAMILIES):  # cover each family once
        name, fam, s = G.FAMILIES[seed]
        inst.update(family=name, fam=fam, s=s)
    k, v = G.instance_kv(inst)
    qc = planner.kv_query(k, v)
    rel.planner_set(torch.from_numpy(__import__("synth").mlp_params(seed)).cuda())
    q = oracle.kv_query(k.cpu().numpy(), v.cpu().numpy())
    ek, ea = oracle.groupby(q)
    for flags in (rel.PLAN_LEARNED | rel.PLAN_SKETCH, rel.PLAN_EXACT | rel.PLAN_SKETCH):
        keys, aggs, plan = rel.groupby_auto(qc, flags=flags)
        gk, ga = canon_groupby(keys, aggs)
        assert np.array_equal(gk, ek) and np.array_equal(ga, ea)


@pytest.mark.skipif(not os.path.exists(planner.DEFAULT_WEIGHTS), reason="no trained network")
def test_trained_network_beats_exact_prepass():
    r = planner.evaluate(range(2_000_000, 2_000_024), with_labels=False, log_every=0)
    assert r["mismatches"] == 0
    assert r["speedup_vs_exact"] > 1.0, r["ms_total"]
