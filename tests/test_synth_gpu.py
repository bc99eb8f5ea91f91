"""The GPU input generator (synth/gen_gpu.cu): its uniform family and its
values are the host generator's streams bit for bit; the Zipf family matches
its target probabilities; the clustered family has the stated run lengths."""
import math

import numpy as np
import pytest
import torch

import synth
from synth import gpu as G

pytestmark = pytest.mark.gpu


def test_uniform_family_equals_host_stream():
    n, D, seed = 300_001, 12345, 77
    k, v = G.kv(0, 0.0, n, D, seed)
    np.testing.assert_array_equal(k.cpu().numpy(), synth.uniform_mixed(n, 1, D, seed, synth.TAG_KEY))
    np.testing.assert_array_equal(v.cpu().numpy(),
                                  synth.uniform(n, -10**6, 10**6, seed, synth.TAG_VAL))


@pytest.mark.parametrize("s", [0.5, 1.0, 1.5])
def test_zipf_frequencies(s):
    n, D = 4_000_000, 1000
    k, _ = G.kv(1, s, n, D, seed=5)
    k = k.cpu().numpy()
    ranks = np.arange(1, D + 1)
    keys = np.array([synth.mix64_signed(int(r)) for r in ranks], dtype=np.int64)
    order = np.argsort(keys)
    pos = np.searchsorted(keys[order], k)
    assert np.all(keys[order][np.minimum(pos, D - 1)] == k), "key outside the domain"
    counts = np.bincount(order[pos], minlength=D).astype(np.float64)
    p = ranks.astype(np.float64) ** -s
    p /= p.sum()
    # the 20 most likely ranks within 5 standard deviations each
    for r in range(20):
        sd = math.sqrt(n * p[r] * (1 - p[r]))
        assert abs(counts[r] - n * p[r]) < 5 * sd, (r, counts[r], n * p[r])
    # and the whole distribution by a chi-square statistic (D - 1 dof)
    chi2 = ((counts - n * p) ** 2 / (n * p)).sum()
    assert chi2 < D + 6 * math.sqrt(2 * D)


def test_clustered_runs():
    n, D = 2_000_000, 10**8
    k, _ = G.kv(2, 0.0, n, D, seed=9)
    k = k.cpu().numpy()
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    runs = np.diff(np.r_[starts, n])
    # geometric(1/64): mean 64, sd ~ 63.5; runs merge only when two adjacent
    # runs draw the same rank (probability ~1e-8 here)
    assert abs(runs.mean() - 64) < 3
    assert runs.max() <= 4096
    # median of geometric(1/64) on {1, 2, ...}: ceil(ln 2 / -ln(63/64)) = 45
    assert abs(np.median(runs) - 45) <= 3


def test_determinism_and_empty():
    a, _ = G.kv(1, 1.0, 100_000, 10**7, seed=3)
    b, _ = G.kv(1, 1.0, 100_000, 10**7, seed=3)
    assert torch.equal(a, b)
    e, f = G.kv(2, 0.0, 0, 10, seed=3)
    assert e.numel() == 0 and f.numel() == 0



def test_join_sides_equal_host_streams():
    bk, bp, pk = G.join_sides(30_001, 200_003, seed=11)
    hk, hp = synth.join_build(30_001, seed=11)
    hq, _ = synth.join_probe(200_003, 30_001, seed=11)
    np.testing.assert_array_equal(bk.cpu().numpy(), hk)
    np.testing.assert_array_equal(bp.cpu().numpy(), hp)
    np.testing.assert_array_equal(pk.cpu().numpy(), hq)
