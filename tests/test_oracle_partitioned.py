"""The multi-core CPU baseline (the oracle run on hash partitions of the
rows, one thread each) gives exactly the single-threaded oracle's result.
CPU only."""
import numpy as np
import pytest

import oracle
import synth
from oracle import partitioned as P

from test_oracle_groupby import rand_query


def same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
        assert x.dtype == y.dtype


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("threads", [2, 3, 8])
def test_groupby_random_queries(seed, threads):
    rng = np.random.default_rng(1000 + seed)
    q = rand_query(rng, int(rng.integers(1, 3000)))
    same(P.groupby(q, threads=threads), oracle.groupby(q))


def test_groupby_workloads():
    li = oracle.lineitem_query(synth.lineitem(50_000, seed=3))
    same(P.groupby(li, threads=5), oracle.groupby(li))
    k, v = synth.zipf_kv(200_000, seed=4)
    q = oracle.kv_query(k, v)
    same(P.groupby(q, threads=7), oracle.groupby(q))
    k4, v4 = synth.few_keys_kv(100_000, n_keys=4, seed=5)
    q4 = oracle.kv_query(k4, v4)
    same(P.groupby(q4, threads=16), oracle.groupby(q4))


def test_groupby_unsorted_is_a_permutation():
    k, v = synth.zipf_kv(50_000, seed=6)
    q = oracle.kv_query(k, v)
    gk, ga = P.groupby(q, threads=4, sort=False)
    ek, ea = oracle.groupby(q)
    o = np.argsort(gk)
    same((gk[o], ga[:, o]), (ek, ea))


def test_groupby_empty_and_filtered_out():
    q = oracle.kv_query(np.empty(0, np.int64), np.empty(0, np.int64))
    gk, ga = P.groupby(q, threads=4)
    assert gk.size == 0 and ga.shape == (4, 0)
    k = np.arange(100, dtype=np.int64)
    q = {"cols": [k, k], "keys": [0], "preds": [(1, 1000, 2000)], "aggs": [("sum", 1, [])]}
    gk, ga = P.groupby(q, threads=4)
    assert gk.size == 0 and ga.shape == (1, 0)


@pytest.mark.parametrize("threads", [2, 5, 8])
def test_join_with_duplicates(threads):
    rng = np.random.default_rng(threads)
    bk = rng.integers(-20, 20, 3000).astype(np.int64)
    bp = rng.integers(-(2**63), 2**63 - 1, 3000, dtype=np.int64)
    pk = rng.integers(-25, 25, 7000).astype(np.int64)
    same(P.join(bk, bp, pk, threads=threads), oracle.join(bk, bp, pk))


def test_join_workload_and_edges():
    bk, bp = synth.join_build(20_000, seed=1)
    pk, _ = synth.join_probe(100_000, 20_000, seed=1)
    same(P.join(bk, bp, pk, threads=6), oracle.join(bk, bp, pk))
    e = np.empty(0, np.int64)
    same(P.join(e, e, pk, threads=4), oracle.join(e, e, pk))
    same(P.join(bk, bp, e, threads=4), oracle.join(bk, bp, e))


def test_partition_depends_on_key_values_only():
    a = np.array([5, -1, 5, 7, -1], dtype=np.int64)
    b = np.array([1, 2, 1, 1, 2], dtype=np.uint8)
    p = P.partition_of([a, b], 8)
    assert p[0] == p[2] and p[1] == p[4]
    assert p.min() >= 0 and p.max() < 8
    # int32 and int64 columns holding the same values hash alike
    assert np.array_equal(P.partition_of([a.astype(np.int32)], 8), P.partition_of([a], 8))
