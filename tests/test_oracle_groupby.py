"""Pins for the oracle's filtered group-by (CPU only).

The oracle is checked against things other than itself: a pure-Python
brute force written from the definition (dict of groups, Python big ints
reduced mod 2^64), numpy whole-column formulations, invariants that hold for
any correct group-by, and special cases that reduce to a library routine.
Each check is chosen so that a plausible slip in oracle.cpp -- a dropped
factor, a sign flip in c + s*x, an unsigned min, a wrong key packing order,
a missed predicate bound, a lost wrap -- fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import synth

M64 = (1 << 64) - 1


def s64(x):
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def brute_groupby(q):
    """Definition, row by row, in Python integers."""
    cols = [c.tolist() for c in q["cols"]]
    dts = [c.dtype for c in q["cols"]]
    n = len(cols[0]) if cols else 0
    groups = {}
    for i in range(n):
        if not all(lo <= cols[c][i] <= hi for c, lo, hi in q.get("preds", [])):
            continue
        if len(q["keys"]) == 1:
            key = cols[q["keys"][0]][i]
        else:
            key = 0
            for c in q["keys"]:
                w = {np.dtype(np.uint8): 8, np.dtype(np.int32): 32}[dts[c]]
                key = key * (1 << w) + (cols[c][i] % (1 << w))
            key = s64(key)
        g = groups.setdefault(key, [[] for _ in q["aggs"]])
        for a, (op, base, fs) in enumerate(q["aggs"]):
            v = cols[base][i]
            for fc, c, s in fs:
                v = v * (c + s * cols[fc][i])
            g[a].append(s64(v))
    keys = sorted(groups)
    out = np.zeros((len(q["aggs"]), len(keys)), dtype=np.int64)
    for j, k in enumerate(keys):
        for a, (op, _, _) in enumerate(q["aggs"]):
            vals = groups[k][a]
            r = {"sum": lambda: s64(sum(vals)), "count": lambda: len(vals),
                 "min": lambda: min(vals), "max": lambda: max(vals)}[op]()
            out[a, j] = r
    return np.array(keys, dtype=np.int64), out


def rand_query(rng, n):
    """Random small query over mixed column types."""
    cols = [
        rng.integers(0, 4, n).astype(np.uint8),
        rng.integers(-3, 3, n).astype(np.int32),
        rng.integers(-(2**62), 2**62, n, dtype=np.int64) * rng.integers(1, 3, n),
        rng.integers(-50, 50, n).astype(np.int64),
        rng.integers(0, 256, n).astype(np.uint8),
    ]
    nk = int(rng.integers(1, 3))
    keys = [0] if nk == 1 else [0, 1]
    if rng.random() < 0.3:
        keys = [int(rng.choice([1, 2, 3]))]
    preds = []
    if rng.random() < 0.7:
        preds.append((3, int(rng.integers(-50, 0)), int(rng.integers(0, 50))))
    if rng.random() < 0.3:
        preds.append((4, 10, 200))
    aggs = []
    for op in ["sum", "count", "min", "max"]:
        fs = []
        for _ in range(int(rng.integers(0, 3))):
            fs.append((int(rng.choice([1, 3, 4])), int(rng.integers(-200, 200)),
                       int(rng.choice([-1, 1, 3]))))
        aggs.append((op, int(rng.choice([2, 3, 1])), fs))
    rng.shuffle(aggs)
    return {"cols": cols, "keys": keys, "preds": preds, "aggs": aggs}


@pytest.mark.parametrize("seed", range(40))
def test_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 300))
    q = rand_query(rng, n)
    k, a = oracle.groupby(q)
    bk, ba = brute_groupby(q)
    np.testing.assert_array_equal(k, bk)
    np.testing.assert_array_equal(a, ba)


def test_all_subsets_tiny():
    """Every subset of a 10-row table (as a predicate mask) against brute force."""
    rng = np.random.default_rng(7)
    base = {
        "k": rng.integers(0, 3, 10).astype(np.int64),
        "v": rng.integers(-9, 9, 10).astype(np.int64),
    }
    for mask in range(1 << 10):
        sel = np.array([(mask >> i) & 1 for i in range(10)], dtype=np.int32)
        q = {"cols": [base["k"], base["v"], sel], "keys": [0], "preds": [(2, 1, 1)],
             "aggs": [("sum", 1, []), ("count", 1, []), ("min", 1, []), ("max", 1, [])]}
        k, a = oracle.groupby(q)
        bk, ba = brute_groupby(q)
        assert np.array_equal(k, bk) and np.array_equal(a, ba), mask


def test_lineitem_invariants_and_closed_forms():
    li = synth.lineitem(200_000, seed=3)
    q = oracle.lineitem_query(li)
    k, a = oracle.groupby(q)
    keep = li["date"] <= 2430
    # key packing: (flag << 8) | status, the 6 combinations in ascending order
    np.testing.assert_array_equal(k, [0, 1, 256, 257, 512, 513])
    # sum of counts == filtered rows
    assert a[4].sum() == keep.sum()
    # per-group sums against a numpy whole-column formulation
    price = li["price"][keep]
    disc = li["disc"][keep]
    tax = li["tax"][keep]
    disc_price = price * (100 - disc)
    charge = disc_price * (100 + tax)
    gid = li["flag"][keep].astype(np.int64) * 256 + li["status"][keep]
    for col, agg in [(li["qty"][keep], a[0]), (price, a[1]), (disc_price, a[2]),
                     (charge, a[3])]:
        ref = np.array([col[gid == g].sum() for g in k], dtype=np.int64)
        np.testing.assert_array_equal(agg, ref)
    cnt = np.array([(gid == g).sum() for g in k])
    np.testing.assert_array_equal(a[4], cnt)


def test_sum_invariants_zipf():
    keys, vals = synth.zipf_kv(300_000, seed=5, n_ranks=100_000)
    k, a = oracle.groupby(oracle.kv_query(keys, vals))
    assert np.all(np.diff(k) > 0)  # strictly ascending, unique
    assert a[1].sum() == len(keys)
    assert int(a[0].sum()) == int(vals.sum())
    assert a[2].min() == vals.min() and a[3].max() == vals.max()
    assert np.all(a[2] <= a[3])
    uk = np.unique(keys)
    np.testing.assert_array_equal(k, uk)
    # per-group count against np.unique's counts
    _, cnt = np.unique(keys, return_counts=True)
    np.testing.assert_array_equal(a[1], cnt)


def test_one_group_reduces_to_library():
    rng = np.random.default_rng(11)
    v = rng.integers(-(10**12), 10**12, 5000)
    k = np.full(5000, -77, dtype=np.int64)
    kk, a = oracle.groupby(oracle.kv_query(k, v))
    assert kk.tolist() == [-77]
    assert a[:, 0].tolist() == [int(v.sum()), 5000, int(v.min()), int(v.max())]


def test_all_distinct_keys_reproduce_rows():
    rng = np.random.default_rng(12)
    k = rng.permutation(np.arange(-500, 1500, dtype=np.int64))
    v = rng.integers(-100, 100, len(k))
    kk, a = oracle.groupby(oracle.kv_query(k, v))
    order = np.argsort(k)
    np.testing.assert_array_equal(kk, k[order])
    for row in (0, 2, 3):
        np.testing.assert_array_equal(a[row], v[order])
    assert np.all(a[1] == 1)


def test_predicate_bounds_inclusive_and_empty():
    d = np.array([0, 2430, 2431, 2526], dtype=np.int32)
    k = np.zeros(4, np.uint8)
    q = {"cols": [k, d], "keys": [0], "preds": [(1, -(2**31), 2430)],
         "aggs": [("count", 1, [])]}
    assert oracle.groupby(q)[1].tolist() == [[2]]
    q["preds"] = [(1, 3000, 4000)]
    kk, a = oracle.groupby(q)
    assert kk.size == 0 and a.shape == (1, 0)
    q["cols"] = [k[:0], d[:0]]
    kk, a = oracle.groupby(q)
    assert kk.size == 0


def test_wraparound_mod_2_64():
    v = np.array([2**62, 2**62, 2**62, -(2**63)], dtype=np.int64)
    k = np.zeros(4, np.int64)
    q = {"cols": [k, v], "keys": [0], "preds": [],
         "aggs": [("sum", 1, []), ("sum", 1, [(1, 0, 2)])]}
    _, a = oracle.groupby(q)
    assert a[0, 0] == s64(3 * 2**62 - 2**63)
    assert a[1, 0] == s64(sum(2 * x * x for x in v.tolist()))


def test_min_max_signed_and_extremes():
    v = np.array([-1, 5, np.iinfo(np.int64).min, np.iinfo(np.int64).max], dtype=np.int64)
    k = np.array([1, 1, 2, 2], dtype=np.int64)
    _, a = oracle.groupby(oracle.kv_query(k, v, ops=("min", "max")))
    assert a.tolist() == [[-1, np.iinfo(np.int64).min], [5, np.iinfo(np.int64).max]]


def test_key_sentinel_values_are_ordinary_keys():
    k = np.array([np.iinfo(np.int64).min, 0, np.iinfo(np.int64).max, np.iinfo(np.int64).min],
                 dtype=np.int64)
    v = np.array([1, 2, 3, 4], dtype=np.int64)
    kk, a = oracle.groupby(oracle.kv_query(k, v, ops=("sum", "count")))
    assert kk.tolist() == [np.iinfo(np.int64).min, 0, np.iinfo(np.int64).max]
    assert a.tolist() == [[5, 2, 3], [2, 1, 1]]


def test_packed_key_widths():
    """Two i32 key columns pack into 64 bits: first column high word."""
    a = np.array([-1, 0, 1], dtype=np.int32)
    b = np.array([-1, 7, 0], dtype=np.int32)
    q = {"cols": [a, b], "keys": [0, 1], "preds": [], "aggs": [("count", 0, [])]}
    kk, _ = oracle.groupby(q)
    expect = sorted(s64(((x & 0xFFFFFFFF) << 32) | (y & 0xFFFFFFFF))
                    for x, y in zip(a.tolist(), b.tolist()))
    assert kk.tolist() == expect
