"""Pins for the oracle's equi-join (CPU only).

Checked against a pure-Python nested loop, the histogram dot product
|pairs| = sum_k h_build(k) * h_probe(k), and the generator's own record of
which probe rows were drawn from the build side.
"""
import numpy as np
import pytest

import oracle
import synth


def brute_join(bk, bp, pk):
    out = []
    for i, x in enumerate(pk.tolist()):
        for j, y in enumerate(bk.tolist()):
            if x == y:
                out.append((i, j, int(bp[j])))
    return out


def hist_dot(bk, pk):
    ub, cb = np.unique(bk, return_counts=True)
    up, cp = np.unique(pk, return_counts=True)
    common, ib, ip = np.intersect1d(ub, up, return_indices=True)
    return int((cb[ib].astype(np.int64) * cp[ip]).sum())


@pytest.mark.parametrize("seed", range(25))
def test_matches_nested_loop_with_duplicates(seed):
    rng = np.random.default_rng(100 + seed)
    nb, npr = int(rng.integers(0, 60)), int(rng.integers(0, 80))
    dom = int(rng.integers(1, 20))
    bk = rng.integers(-dom, dom, nb).astype(np.int64)
    if nb and rng.random() < 0.3:
        bk[0] = np.iinfo(np.int64).min
    pk = rng.integers(-dom, dom, npr).astype(np.int64)
    if npr and rng.random() < 0.3:
        pk[-1] = np.iinfo(np.int64).min
    bp = rng.integers(-(2**63), 2**63 - 1, nb, dtype=np.int64)
    pi, bi, pay = oracle.join(bk, bp, pk)
    got = list(zip(pi.tolist(), bi.tolist(), pay.tolist()))
    assert got == brute_join(bk, bp, pk)
    assert len(got) == hist_dot(bk, pk) == oracle.join_count(bk, pk)


def test_hash_branch_matches_nested_branch():
    """Sizes past the nested-loop limit take the multimap branch; same bag."""
    rng = np.random.default_rng(5)
    bk = rng.integers(0, 3000, 5000).astype(np.int64)  # duplicates
    bp = np.arange(5000, dtype=np.int64) * 7
    pk = rng.integers(0, 4000, 4000).astype(np.int64)
    pi, bi, pay = oracle.join(bk, bp, pk)  # 2e7 > 2^24: hash branch
    assert len(pi) == hist_dot(bk, pk)
    # sorted by (probe, build), each pair a real match, payload gathered
    order = np.lexsort((bi, pi))
    assert np.array_equal(order, np.arange(len(pi)))
    assert np.all(pk[pi] == bk[bi]) and np.all(pay == bp[bi])
    # compare against the nested branch on a slice that stays below 2^24
    sub = slice(0, 3000)
    pi2, bi2, pay2 = oracle.join(bk[:5000], bp[:5000], pk[sub])  # 1.5e7 <= 2^24
    keep = pi < 3000
    assert np.array_equal(pi2, pi[keep]) and np.array_equal(bi2, bi[keep])


def test_generator_closed_form():
    """Unique build keys, 90% present probes: every present row matches once,
    every absent row never; payload is the build row's payload."""
    nb, npr = 20_000, 300_000
    bk, bp = synth.join_build(nb, seed=9)
    pk, present = synth.join_probe(npr, nb, seed=9)
    pi, bi, pay = oracle.join(bk, bp, pk)
    assert len(pi) == int(present.sum())
    assert np.array_equal(pi, np.flatnonzero(present))
    assert np.all(pk[pi] == bk[bi]) and np.all(pay == bp[bi])
    assert oracle.join_count(bk, pk) == len(pi)


def test_empty_sides():
    e = np.empty(0, np.int64)
    k = np.arange(5, dtype=np.int64)
    for b, p in [(e, k), (k, e), (e, e)]:
        pi, bi, pay = oracle.join(b, np.zeros(len(b), np.int64), p)
        assert len(pi) == 0
