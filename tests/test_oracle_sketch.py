"""Pins for the oracle's sample sketch (CPU only): a pure-Python statement of
the same definition, the published SplitMix64 output the HLL hash is, and
the HyperLogLog error bound of Flajolet et al. (2007)."""
import math
from collections import Counter

import numpy as np
import pytest

import oracle
import synth


def py_sketch(q):
    cols = [c.tolist() for c in q["cols"]]
    n = len(cols[0])
    S = min(n, 4096)
    kept, blocks = [], []
    for j in range(S):
        row = j if n <= 4096 else (j // 64) * (n - 64) // 63 + (j % 64)
        if not all(lo <= cols[c][row] <= hi for c, lo, hi in q.get("preds", [])):
            continue
        assert len(q["keys"]) == 1
        kept.append(cols[q["keys"][0]][row])
        blocks.append(j // 64)
    regs = [0] * 256
    for k in kept:
        h = synth.mix64(k % (1 << 64))
        rest = (h << 8) % (1 << 64)
        rank = 57 if rest == 0 else 64 - rest.bit_length() + 1
        regs[h >> 56] = max(regs[h >> 56], rank)
    cnt = Counter(kept)
    runs = sum(1 for i in range(len(kept))
               if i == 0 or blocks[i] != blocks[i - 1] or kept[i] != kept[i - 1])
    top = sorted(cnt.items(), key=lambda kv: (-kv[1], kv[0]))[:32]
    return {"sample_rows": S, "kept": len(kept), "ndv": len(cnt),
            "singletons": sum(1 for v in cnt.values() if v == 1), "runs": runs,
            "key_min": min(kept) if kept else 0, "key_max": max(kept) if kept else 0,
            "top": top, "hll": regs}


def check(q):
    s = oracle.sketch(q)
    b = py_sketch(q)
    for f in ("sample_rows", "kept", "ndv", "singletons", "runs", "key_min", "key_max"):
        assert s[f] == b[f], f
    got_top = [(int(k), int(c)) for k, c in zip(s["top_key"], s["top_count"]) if c > 0]
    assert got_top == b["top"]
    assert s["hll"].tolist() == b["hll"]
    return s


@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 4095, 4096, 4097, 50_000])
def test_matches_python_definition(n):
    rng = np.random.default_rng(n)
    k = rng.integers(-50, 50, n).astype(np.int64)
    v = rng.integers(0, 10, n).astype(np.int64)
    check({"cols": [k, v], "keys": [0], "preds": [(1, 2, 7)], "aggs": [("count", 0, [])]})


def test_clustered_runs_and_zipf_top():
    keys, vals = synth.zipf_kv(300_000, seed=4, n_ranks=1000)
    s = check(oracle.kv_query(keys, vals))
    assert s["top_key"][0] == synth.mix64_signed(1)  # rank 1 is the most frequent
    # runs of 64 equal keys; n = 64 + 63 * 128 puts every window start on a
    # run boundary (start = 128 w), so each window holds exactly one run
    runs = np.repeat(np.arange(127, dtype=np.int64), 64)
    assert len(runs) == 64 + 63 * 128
    s = check(oracle.kv_query(runs, runs))
    assert s["runs"] == 64
    assert s["features"][256 + 6] == 64.0


def test_special_cases():
    const = np.full(10_000, 7, np.int64)
    s = check(oracle.kv_query(const, const))
    assert s["ndv"] == 1 and s["singletons"] == 0 and s["features"][256 + 3] == 1.0
    iota = np.arange(-3000, 3000, dtype=np.int64)
    s = check(oracle.kv_query(iota, iota))
    assert s["ndv"] == s["singletons"] == s["kept"] == 4096
    # the first window starts at row 0 and the last ends at row 5999
    assert s["key_min"] == -3000 and s["key_max"] == 2999
    assert s["features"][256 + 2] == pytest.approx(math.log2(6000))
    q = oracle.kv_query(iota, iota)
    q["preds"] = [(1, 10**9, 10**9 + 1)]
    s = check(q)
    assert s["kept"] == 0 and s["ndv"] == 0 and not s["hll"].any()


def test_features_layout():
    li = synth.lineitem(100_000, seed=2)
    q = oracle.lineitem_query(li)
    cols = q["cols"]
    s = oracle.sketch(q)
    f = s["features"]
    assert f.shape == (264,)
    assert np.allclose(f[:256], s["hll"] / 57.0)
    assert f[256] == pytest.approx(math.log2(100_000))
    assert f[263] == 16 / 64  # two u8 key columns packed
    assert s["ndv"] == 6


@pytest.mark.parametrize("ndv", [10, 300, 3000])
def test_hll_within_flajolet_bound(ndv):
    """p = 8: standard error 1.04 / 16; 3 sigma holds for these seeds."""
    keys = synth.uniform_mixed(4096, 1, ndv, seed=ndv, tag=5)
    s = oracle.sketch(oracle.kv_query(keys, keys))
    est = oracle.hll_estimate(s["hll"])
    assert abs(est - s["ndv"]) <= 3 * 1.04 / 16 * s["ndv"] + 1


def test_key_hll_pins():
    """The full-data HyperLogLog: the clz helper on exact powers and extremes;
    registers equal to a per-key pure-Python restatement on a small input; the
    estimate within three standard errors (3 x 1.04 / 64) of the exact count
    for large inputs and close to it (linear counting) for small ones."""
    import numpy as np

    import oracle
    import synth

    x = np.array([0, 1, 2, 3, (1 << 63), (1 << 63) + 5, (1 << 40), (1 << 64) - 1], np.uint64)
    assert oracle._clz64(x).tolist() == [64, 63, 62, 62, 0, 0, 23, 0]
    M = (1 << 64) - 1

    def fmix(k):
        k ^= k >> 33
        k = (k * 0xFF51AFD7ED558CCD) & M
        k ^= k >> 33
        k = (k * 0xC4CEB9FE1A85EC53) & M
        return k ^ (k >> 33)

    keys = synth.uniform(3000, -(2**62), 2**62, seed=3, tag=1)
    keys[:5] = [0, -1, np.iinfo(np.int64).min, np.iinfo(np.int64).max, 7]
    want = [0] * 4096
    for key in keys.tolist():
        h = fmix((key & M) ^ (1 << 63))
        rest = (h << 12) & M
        rank = 53 if rest == 0 else 64 - rest.bit_length() + 1
        want[h >> 52] = max(want[h >> 52], rank)
    regs, _ = oracle.key_hll(keys)
    assert regs.tolist() == want
    # int32 keys sign-extend
    k32 = synth.uniform(5000, -1000, 1000, seed=4, tag=2, dtype=np.int32)
    assert np.array_equal(oracle.key_hll(k32)[0], oracle.key_hll(k32.astype(np.int64))[0])
    for n, dom in ((2_000_000, 10**7), (300_000, 10**12), (800, 10**6)):
        k = synth.uniform(n, 0, dom, seed=n, tag=3)
        true = np.unique(k).size
        _, est = oracle.key_hll(k)
        tol = 3 * 1.04 / 64 if true > 5 * 4096 else 0.02
        assert abs(est - true) <= tol * true, (n, true, est)
