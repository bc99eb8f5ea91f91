"""The operators sharded over several GPUs, one process per GPU (torch.distributed).

Group-by: rows are partitioned across ranks as they come.  Every rank
aggregates its own rows (rel.groupby), splits its partial groups by owner rank
in the library (rel.shard_split: owner = a hash of the key), and one
all-to-all exchange sends every partial group to its owner, which merges the
partials of each of its keys with a second group-by: SUM of sums, SUM of
counts, MIN of minima, MAX of maxima.  Those merges are exact in int64
arithmetic (wrap-around included), so the union of the ranks' results is the
unsharded result bit for bit, and every key ends up on exactly one rank.

Join: the build side is small enough to replicate (1e6 x 16 bytes): the rank
that holds it broadcasts it, every rank builds the same table and probes its
own rows of the probe side; a rank's pairs carry local probe indices, and an
all-gather of the pair counts gives each rank the offset of its pairs in the
concatenated output.

The exchange is plain data movement (torch.distributed all-to-all of the
per-owner ranges); every arithmetic step runs in the library's kernels.  This
module is the multi-GPU path: it is exercised with CPU (gloo) ranks in the
tests, where the per-rank compute is supplied by the test, and it has not
been measured on a multi-GPU machine.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

# partial aggregate op -> the op that merges partials of one key
MERGE = {"sum": "sum", "count": "sum", "min": "min", "max": "max"}


def merge_ops(ops) -> list:
    """Aggregate ops that combine partial results of `ops`."""
    return [MERGE[o] for o in ops]


def _world(group):
    return dist.get_world_size(group), dist.get_rank(group)


def exchange(keys: torch.Tensor, words: list, counts: list, group=None):
    """All-to-all of partial groups that are already grouped by owner:
    keys / words hold owner 0's groups first, then owner 1's, ...; counts[r]
    is how many go to rank r.  Returns the (keys, [words]) this rank owns,
    from every rank, unmerged."""
    world, _ = _world(group)
    if len(counts) != world:
        raise ValueError("one count per rank")
    send = torch.tensor(counts, dtype=torch.int64)
    recv = torch.empty(world, dtype=torch.int64)
    if keys.is_cuda:
        send, recv = send.to(keys.device), recv.to(keys.device)
    dist.all_to_all_single(recv, send, group=group)
    rc = [int(x) for x in recv.tolist()]
    out_k = torch.empty(sum(rc), dtype=keys.dtype, device=keys.device)
    dist.all_to_all_single(out_k, keys.contiguous(), output_split_sizes=rc,
                           input_split_sizes=list(counts), group=group)
    out_w = []
    for w in words:
        o = torch.empty(sum(rc), dtype=w.dtype, device=w.device)
        dist.all_to_all_single(o, w.contiguous(), output_split_sizes=rc,
                               input_split_sizes=list(counts), group=group)
        out_w.append(o)
    return out_k, out_w


def groupby_sharded(q_local: dict, group=None, flags: int | None = None):
    """The sharded group-by on this rank's GPU: local aggregation, split by
    owner, exchange, merge.  q_local: this rank's rows, as for rel.groupby
    (one key column; aggregates sum / count / min / max).  Returns the groups
    this rank owns (keys, [aggs])."""
    from . import rel

    world, _ = _world(group)
    ops = [a[0] for a in q_local["aggs"]]
    f = rel.PLAN_EXACT | rel.PLAN_SKETCH if flags is None else flags
    keys, aggs = rel.groupby(q_local, flags=f)
    out_k, out_w, counts = rel.shard_split(keys.contiguous(), [a.contiguous() for a in aggs],
                                           world)
    rk, rw = exchange(out_k, out_w, counts, group)
    if rk.numel() == 0:
        return rk, [torch.empty(0, dtype=torch.int64, device=rk.device) for _ in ops]
    merged = {"cols": [rk, *rw], "keys": [0], "preds": [],
              "aggs": [(m, 1 + i, []) for i, m in enumerate(merge_ops(ops))]}
    return rel.groupby(merged, flags=f)


def join_sharded(build_keys, build_payload, probe_local: torch.Tensor, src: int = 0,
                 group=None):
    """The sharded join on this rank's GPU: the build side is broadcast from
    rank src (every rank passes tensors of the same shape; only src's contents
    matter), every rank probes its own probe rows.  Returns (probe_idx local to
    this rank's rows, build_idx, payload, offset of this rank's pairs in the
    concatenation of all ranks' pairs in rank order)."""
    from . import rel

    dist.broadcast(build_keys, src, group=group)
    dist.broadcast(build_payload, src, group=group)
    t = rel.JoinTable(build_keys, build_payload)
    pi, bi, pay = t.probe(probe_local)
    return (pi, bi, pay) + (pair_offset(pi.numel(), group, probe_local.device),)


def pair_offset(n_pairs: int, group=None, device=None) -> int:
    """Exclusive prefix over ranks of their pair counts (rank order)."""
    world, rank = _world(group)
    mine = torch.tensor([n_pairs], dtype=torch.int64, device=device)
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    return int(sum(int(x.item()) for x in every[:rank]))
