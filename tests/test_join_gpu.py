"""GPU parity of the hash equi-join (build, count, probe + payload gather)
against the oracle: bit-exact pair sets after sorting by (probe_idx,
build_idx), at small sizes with duplicate and INT64_MIN keys, and at the
full 10^6 x 1.6*10^7 size the benchmark times."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2608_13696_gb300 import rel

from gpu_util import canon_join, cuda

pytestmark = pytest.mark.gpu


def gpu_join(bk, bp, pk, capacity=None):
    t = rel.JoinTable(cuda(bk), cuda(bp))
    pkc = cuda(pk)
    cnt = t.count(pkc)
    pi, bi, pay = t.probe(pkc, capacity=capacity)
    torch.cuda.synchronize()
    return cnt, canon_join(pi, bi, pay)


def assert_same(bk, bp, pk, capacity=None):
    cnt, (pi, bi, pay) = gpu_join(bk, bp, pk, capacity)
    epi, ebi, epay = oracle.join(bk, bp, pk)
    assert cnt == len(epi)
    np.testing.assert_array_equal(pi, epi)
    np.testing.assert_array_equal(bi, ebi)
    np.testing.assert_array_equal(pay, epay)


@pytest.mark.parametrize("seed", range(10))
def test_duplicates_and_sentinel(seed):
    rng = np.random.default_rng(seed)
    nb, npr = int(rng.integers(1, 3000)), int(rng.integers(1, 20000))
    dom = int(rng.integers(1, 500))
    bk = rng.integers(-dom, dom, nb).astype(np.int64)
    pk = rng.integers(-dom, dom, npr).astype(np.int64)
    bk[:: max(1, nb // 5)] = np.iinfo(np.int64).min
    pk[:: max(1, npr // 7)] = np.iinfo(np.int64).min
    bp = rng.integers(-(2**63), 2**63 - 1, nb, dtype=np.int64)
    assert_same(bk, bp, pk)


def test_generated_medium():
    bk, bp = synth.join_build(20_000, seed=1)
    pk, present = synth.join_probe(300_001, 20_000, seed=1)
    assert_same(bk, bp, pk)


def test_full_size_1m_x_16m():
    bk, bp = synth.join_build(1_000_000, seed=0)
    pk, present = synth.join_probe(16_000_000, 1_000_000, seed=0)
    cnt, (pi, bi, pay) = gpu_join(bk, bp, pk)
    # closed form from the generator: each present row matches exactly once
    assert cnt == len(pi) == int(present.sum())
    np.testing.assert_array_equal(pi, np.flatnonzero(present))
    np.testing.assert_array_equal(pk[pi], bk[bi])
    np.testing.assert_array_equal(pay, bp[bi])
    epi, ebi, epay = oracle.join(bk, bp, pk)
    np.testing.assert_array_equal(bi, ebi)


def test_capacity_retry_and_status():
    bk = np.repeat(np.arange(50, dtype=np.int64), 3)
    bp = np.arange(150, dtype=np.int64)
    pk = np.tile(np.arange(60, dtype=np.int64), 4)
    assert_same(bk, bp, pk, capacity=7)


def test_empty_sides():
    e = np.empty(0, np.int64)
    k = np.arange(100, dtype=np.int64)
    for b, p in [(e, k), (k, e)]:
        cnt, (pi, bi, pay) = gpu_join(b, b.copy(), p)
        assert cnt == 0 and len(pi) == 0


def test_unaligned_inputs():
    bk, bp = synth.join_build(5001, seed=3)
    pk, _ = synth.join_probe(40_001, 5000, seed=3)
    t = rel.JoinTable(cuda(bk)[1:], cuda(bp)[1:])
    pi, bi, pay = t.probe(cuda(pk)[1:])
    got = canon_join(pi, bi, pay)
    want = oracle.join(bk[1:], bp[1:], pk[1:])
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("seed", range(40))
def test_unique_keys_small_tables(seed):
    # 1..16 distinct keys in tables of 16 or 32 slots: clustered probe
    # sequences that wrap past the table's end, hits and misses
    rng = np.random.default_rng(100 + seed)
    nb = int(rng.integers(1, 17))
    bk = rng.choice(np.arange(-1000, 1000, dtype=np.int64), nb, replace=False)
    bp = rng.integers(-(2**63), 2**63 - 1, nb, dtype=np.int64)
    pk = np.concatenate([bk, rng.integers(-1200, 1200, 500).astype(np.int64)])
    rng.shuffle(pk)
    assert_same(bk, bp, pk)


def test_unaligned_workspace_rejected():
    L = rel.load()
    bk = cuda(np.arange(100, dtype=np.int64))
    n = L.rel_join_ws_bytes(100)
    ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
    t = rel.JoinTableC()
    st = L.rel_join_build(bk.data_ptr(), bk.data_ptr(), 100, ws.data_ptr() + 8, n, ctypes.byref(t), None)
    assert st == rel.REL_E_INVALID
    assert b"aligned" in L.rel_last_error()
