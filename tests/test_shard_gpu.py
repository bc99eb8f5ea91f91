"""The sharded path's library pieces on one GPU: rel_shard_split regroups
partial groups by owner exactly as the header's owner rule says (checked
against a restatement of the rule), and the whole sharded group-by and join
(local aggregation, split, exchange, merge) run through torch.distributed
with one NCCL rank and match the oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist

import oracle
import synth
from paper_2608_13696_gb300 import rel, sharded

from gpu_util import canon_groupby, canon_join, cuda
from test_sharded_ranks import owner_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [1, 3, 8, 64])
@pytest.mark.parametrize("n", [0, 1, 1000, 300_001])
def test_shard_split_groups_by_owner(world, n):
    k = synth.uniform(n, -10**12, 10**12, seed=world + n, tag=1) if n else np.empty(0, np.int64)
    if n > 10:
        k[::7] = np.iinfo(np.int64).min
    w = [synth.uniform(n, -99, 99, seed=world + n, tag=2 + i) if n else np.empty(0, np.int64)
         for i in range(3)]
    ok, ow, counts = rel.shard_split(cuda(k), [cuda(x) for x in w], world)
    own = owner_of(k, world)
    assert counts == np.bincount(own, minlength=world).tolist()
    ok = ok.cpu().numpy()
    ow = [x.cpu().numpy() for x in ow]
    start = 0
    for r in range(world):
        seg = slice(start, start + counts[r])
        assert (owner_of(ok[seg], world) == r).all()
        start += counts[r]
    # a permutation of the input rows (keys with their words)
    a = np.lexsort([k] + w[::-1])
    b = np.lexsort([ok] + ow[::-1])
    np.testing.assert_array_equal(k[a], ok[b])
    for x, y in zip(w, ow):
        np.testing.assert_array_equal(x[a], y[b])


def test_shard_split_rejects_bad_world():
    k = cuda(np.zeros(4, np.int64))
    with pytest.raises(rel.RelError) as e:
        rel.shard_split(k, [], rel.SHARD_MAX_WORLD + 1)
    assert e.value.status == rel.REL_E_UNSUPPORTED


@pytest.fixture(scope="module")
def nccl_one_rank():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    yield
    dist.destroy_process_group()


def test_sharded_groupby_and_join_one_rank(nccl_one_rank):
    keys, vals = synth.zipf_kv(500_003, seed=51, n_ranks=40_000)
    q = oracle.kv_query(keys, vals)
    qc = dict(q)
    qc["cols"] = [cuda(c) for c in q["cols"]]
    got = canon_groupby(*sharded.groupby_sharded(qc))
    ek, ea = oracle.groupby(q)
    np.testing.assert_array_equal(got[0], ek)
    np.testing.assert_array_equal(got[1], ea)
    bk, bp = synth.join_build(20_000, seed=52)
    pk, _ = synth.join_probe(200_000, 20_000, seed=52)
    pi, bi, pay, off = sharded.join_sharded(cuda(bk), cuda(bp), cuda(pk))
    assert off == 0
    got = canon_join(pi, bi, pay)
    for x, y in zip(got, oracle.join(bk, bp, pk)):
        np.testing.assert_array_equal(x, y)
