"""GPU parity of the batched execution mode (rel_batch_*): every group-by
instance and join partition of a batch equals the oracle bit for bit, for
each tile shape, probe width and placement; CUDA-graph replay; overflow and
capacity flags; the autotuner."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_groupby, canon_join, cuda

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min


def gb_specs():
    """(numpy keys, numpy vals, ops, groups upper bound) per instance."""
    out = []
    k = synth.uniform(300_000, -5, 5, seed=1, tag=3, dtype=np.int32)
    v = synth.uniform(300_000, -10**6, 10**6, seed=1, tag=4)
    out.append((k, v, ["sum", "count"], 11))
    k = synth.uniform_mixed(500_000, 1, 100_000, seed=2, tag=synth.TAG_KEY)
    v = synth.uniform(500_000, -10**6, 10**6, seed=2, tag=synth.TAG_VAL)
    out.append((k, v, ["sum", "count", "min", "max"], 100_000))
    zk, zv = synth.zipf_kv(400_000, seed=3, n_ranks=20_000)
    out.append((zk, zv, ["max", "sum", "min"], 20_000))
    out.append((zk[:0], zv[:0], ["sum", "count"], 1))                        # empty
    s = np.array([I64_MIN] * 7 + list(range(-50, 50)) * 3, dtype=np.int64)  # sentinel key
    out.append((s, s[::-1].copy(), ["sum", "count", "min", "max"], 101))
    k = synth.uniform(1, 0, 0, seed=4, tag=3, dtype=np.int32)                # one row
    out.append((k, np.array([42], np.int64), ["count"], 1))
    k = synth.uniform(70_001, -2**31, 2**31 - 1, seed=5, tag=3, dtype=np.int32)
    v = synth.uniform(70_001, -10**6, 10**6, seed=5, tag=4)
    out.append((k, v, ["min", "max"], 70_001))
    return out


def join_specs():
    out = []
    bk, bp = synth.join_build(50_000, seed=6)
    pk, _ = synth.join_probe(400_000, 50_000, seed=6)
    out.append((bk, bp, pk))
    bk = np.array([5, 5, 7, I64_MIN, I64_MIN, 9, 5], dtype=np.int64)        # duplicates
    bp = np.arange(100, 107, dtype=np.int64)
    pk = np.array([5, 9, I64_MIN, 11, 5, 7, 7, I64_MIN, 0], dtype=np.int64)
    out.append((bk, bp, pk))
    bk, bp = synth.join_build(1000, seed=7)
    out.append((bk, bp, pk[:0]))                                             # empty probe
    pk, _ = synth.join_probe(5000, 1000, seed=8)
    out.append((bk[:0], bp[:0], pk))                                         # empty build
    return out


GB, JN = gb_specs(), join_specs()


def expected_gb(k, v, ops):
    cols = [k, v]
    q = {"cols": cols, "keys": [0], "preds": [], "aggs": [(op, 1, []) for op in ops]}
    return oracle.groupby(q)


EXP_GB = [expected_gb(k, v, ops) for k, v, ops, _ in GB]
EXP_JN = [oracle.join(bk, bp, pk) for bk, bp, pk in JN]


def make_batch(slots_scale=2, capacity=None):
    gs = []
    for (k, v, ops, groups), (ek, _) in zip(GB, EXP_GB):
        slots = 16
        while slots < slots_scale * max(groups, 1):
            slots *= 2
        gs.append({"keys": cuda(k), "vals": cuda(v), "ops": ops, "slots": slots,
                   "est_groups": groups, "capacity": capacity or max(1, len(ek))})
    js = []
    for (bk, bp, pk), e in zip(JN, EXP_JN):
        js.append({"build_keys": cuda(bk), "build_payload": cuda(bp), "probe_keys": cuda(pk),
                   "capacity": capacity or max(1, len(e[0]))})
    return rel.Batch(gs, js)


def check(b):
    counts, flags = b.results()
    ng = len(GB)
    for i, (ek, ea) in enumerate(EXP_GB):
        assert flags[i] == 0, (i, flags[i])
        assert counts[i] == len(ek), i
        k, a = b.groupby_output(i, counts[i])
        gk, ga = canon_groupby(k, a)
        assert np.array_equal(gk, ek), i
        assert np.array_equal(ga, ea), i
    for i, e in enumerate(EXP_JN):
        assert flags[ng + i] == 0
        assert counts[ng + i] == len(e[0])
        got = canon_join(*b.join_output(i, counts[ng + i]))
        for x, y in zip(got, e):
            assert np.array_equal(x, y), i


CONFIGS = [(256, 8, 1, 512), (256, 8, 1, 0), (128, 4, 2, 0), (512, 16, 4, 512), (256, 4, 8, 0),
           (128, 16, 1, 512), (512, 8, 8, 512)]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_batch_matches_oracle(cfg):
    b = make_batch().prepare(cfg)
    b.run()
    check(b)
    b.run()  # a second run starts from zeroed tables again
    check(b)


def test_graph_replay_and_inplace_inputs():
    b = make_batch().prepare((256, 8, 1, 512))
    g = b.capture()
    g.replay()
    check(b)
    # change the first group-by's values in place: the replay sees them
    k, v, ops, _ = GB[0]
    v2 = v * 3 - 7
    b.gspec[0]["vals"].copy_(cuda(v2))
    g.replay()
    counts, _ = b.results()
    ek, ea = expected_gb(k, v2, ops)
    gk, ga = canon_groupby(*b.groupby_output(0, counts[0]))
    assert np.array_equal(gk, ek) and np.array_equal(ga, ea)
    b.gspec[0]["vals"].copy_(cuda(v))


def test_overflow_and_capacity_flags():
    b = make_batch(slots_scale=0).prepare((256, 8, 1, 0))  # 16 slots everywhere
    b.run()
    counts, flags = b.results()
    assert flags[1] & 1 and flags[2] & 1          # 100k / 20k groups in 16 slots
    assert flags[0] == 0 and counts[0] == len(EXP_GB[0][0])  # 11 groups fit
    b = make_batch(capacity=3).prepare((256, 8, 1, 512))
    b.run()
    counts, flags = b.results()
    for i, (ek, _) in enumerate(EXP_GB):
        assert counts[i] == len(ek)
        assert bool(flags[i] & 2) == (len(ek) > 3)
    for i, e in enumerate(EXP_JN):
        assert counts[len(GB) + i] == len(e[0])


def test_autotune_picks_a_candidate():
    b = make_batch()
    cands = [(128, 4, 1, 0), (256, 8, 1, 512), (512, 16, 2, 0), (100, 8, 1, 0)]
    best, ms = b.autotune(cands, reps=2)
    assert best in cands[:3]
    assert ms[(100, 8, 1, 0)] == -1.0                    # invalid block size skipped
    assert all(ms[c] > 0 for c in cands[:3])
    assert ms[best] == min(ms[c] for c in cands[:3])
    b.run()
    check(b)


def test_invalid_config_rejected():
    b = make_batch()
    with pytest.raises(rel.RelError):
        b.prepare((256, 3, 1, 0))
    with pytest.raises(rel.RelError):
        b.prepare((256, 8, 3, 0))
    with pytest.raises(rel.RelError):
        b.prepare((256, 8, 1, 4096))
