"""The sharded path's exchange and merge on CPU ranks (gloo, world 2 and 4):
each rank aggregates its slice of the rows (the oracle stands in for the
GPU group-by here), splits its partial groups by owner with the documented
owner rule, and sharded.exchange (the product code) sends them to their
owners, which merge them with the merge ops (sum of sums, sum of counts, min
of minima, max of maxima).  The union over ranks must equal the unsharded
oracle bit for bit, with every key on exactly one rank -- its owner.  The
join's pair offsets (sharded.pair_offset) are checked the same way against
the unsharded oracle join."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2608_13696_gb300 import sharded

MASK = (1 << 64) - 1
OWNER_MULT = 0xD1B54A32D192ED03


def owner_of(keys: np.ndarray, world: int) -> np.ndarray:
    """floor(h * world / 2^64), h = (k ^ 2^63) * C mod 2^64 (the header's rule)."""
    out = np.empty(len(keys), np.int64)
    for i, k in enumerate(keys.tolist()):
        h = (((k & MASK) ^ (1 << 63)) * OWNER_MULT) & MASK
        out[i] = (h * world) >> 64
    return out


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, vals = synth.zipf_kv(60_000, seed=41, n_ranks=5_000)
        keys[::97] = np.iinfo(np.int64).min
        vals[::13] = np.iinfo(np.int64).max  # sums wrap: the merge must wrap alike
        lo, hi = rank * len(keys) // world, (rank + 1) * len(keys) // world
        ops = ("sum", "count", "min", "max")
        pk, pa = oracle.groupby(oracle.kv_query(keys[lo:hi], vals[lo:hi], ops=ops))
        own = owner_of(pk, world)
        order = np.argsort(own, kind="stable")
        counts = np.bincount(own, minlength=world).tolist()
        rk, rw = sharded.exchange(torch.from_numpy(pk[order]),
                                  [torch.from_numpy(np.ascontiguousarray(a[order])) for a in pa],
                                  counts)
        q = {"cols": [rk.numpy()] + [w.numpy() for w in rw], "keys": [0], "preds": [],
             "aggs": [(m, 1 + i, []) for i, m in enumerate(sharded.merge_ops(ops))]}
        mk, ma = oracle.groupby(q) if rk.numel() else (np.empty(0, np.int64),
                                                       np.empty((4, 0), np.int64))
        # join: build side on rank 0, broadcast; probe slice per rank
        bk, bp = synth.join_build(3_000, seed=42)
        pk2, _ = synth.join_probe(20_000, 3_000, seed=42)
        tb, tp = torch.from_numpy(bk), torch.from_numpy(bp)
        if rank != 0:
            tb.zero_()
            tp.zero_()
        dist.broadcast(tb, 0)
        dist.broadcast(tp, 0)
        plo, phi = rank * len(pk2) // world, (rank + 1) * len(pk2) // world
        pi, bi, pay = oracle.join(tb.numpy(), tp.numpy(), pk2[plo:phi])
        off = sharded.pair_offset(len(pi))
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), mk=mk, ma=ma, pi=pi + plo, bi=bi, pay=pay,
                 off=off, own=owner_of(mk, world) if len(mk) else np.empty(0, np.int64))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_groupby_and_join_equal_unsharded(world, tmp_path):
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    keys, vals = synth.zipf_kv(60_000, seed=41, n_ranks=5_000)
    keys[::97] = np.iinfo(np.int64).min
    vals[::13] = np.iinfo(np.int64).max
    ek, ea = oracle.groupby(oracle.kv_query(keys, vals))
    for r, d in enumerate(res):
        assert (d["own"] == r).all()  # every merged key sits on its owner
    gk = np.concatenate([d["mk"] for d in res])
    ga = np.concatenate([d["ma"] for d in res], axis=1)
    o = np.argsort(gk, kind="stable")
    np.testing.assert_array_equal(gk[o], ek)  # each key exactly once
    np.testing.assert_array_equal(ga[:, o], ea)
    # join: rank r's pairs start at the sum of the lower ranks' counts
    run = 0
    for d in res:
        assert int(d["off"]) == run
        run += len(d["pi"])
    bk, bp = synth.join_build(3_000, seed=42)
    pk2, _ = synth.join_probe(20_000, 3_000, seed=42)
    epi, ebi, epay = oracle.join(bk, bp, pk2)
    gpi = np.concatenate([d["pi"] for d in res])
    gbi = np.concatenate([d["bi"] for d in res])
    gpay = np.concatenate([d["pay"] for d in res])
    o = np.lexsort((gbi, gpi))
    np.testing.assert_array_equal(gpi[o], epi)
    np.testing.assert_array_equal(gbi[o], ebi)
    np.testing.assert_array_equal(gpay[o], epay)


def test_merge_ops():
    assert sharded.merge_ops(["sum", "count", "min", "max"]) == ["sum", "sum", "min", "max"]
