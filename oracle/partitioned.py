"""ORACLE -- test infrastructure, not the product.

The multi-core CPU baseline: the oracle's own single-threaded definitions
(``groupby``, ``join`` in ``oracle.cpp``) run on hash partitions of the rows,
one thread per partition.  ctypes drops the GIL for the length of each
foreign call, so the partitions run on separate cores.

Rows are split by a hash of the group key's columns (group-by) or of the join
key (both join sides), so all rows of one group, and both sides of every
matching pair, land in the same partition: the partition results are
disjoint and their union is the whole result.  No aggregate is merged and no
pair is formed outside the oracle.  Splitting is itself parallel: each
thread orders one contiguous chunk of rows by partition (a stable sort, so
row order within a partition is kept), then each thread gathers one
partition's pieces from every chunk.

Only the CPU-baseline leg of ``bench.py`` and the tests use this module; the
tests check it against the single-threaded oracle.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import groupby as _groupby
from . import join as _join

_MULT = np.uint64(0x9E3779B97F4A7C15)


def default_threads() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 256))


def partition_of(key_cols, n_parts: int) -> np.ndarray:
    """Partition number in [0, n_parts) of every row (uint16, n_parts <=
    65536), a function of the row's values in key_cols only (equal keys,
    equal partition)."""
    if not 1 <= n_parts <= 65536:
        raise ValueError("1 <= n_parts <= 65536")
    h = None
    for c in key_cols:
        x = np.asarray(c).astype(np.uint64)
        if h is None:
            h = x
        else:
            np.bitwise_xor(h, x, out=h)
        np.multiply(h, _MULT, out=h)
    np.right_shift(h, np.uint64(32), out=h)
    np.remainder(h, np.uint64(n_parts), out=h)
    return h.astype(np.uint16)  # a 16-bit key: numpy's stable sort is a radix sort


def _split(cols, key_idx, n_parts: int, pool, n_chunks: int):
    """Per partition, its rows of every column (row order kept) and their row
    numbers: ([cols of partition 0], ...), [row ids of partition 0, ...]."""
    n = len(cols[0])
    bounds = np.linspace(0, n, n_chunks + 1).astype(np.int64)

    def order_chunk(c):
        lo, hi = int(bounds[c]), int(bounds[c + 1])
        part = partition_of([cols[k][lo:hi] for k in key_idx], n_parts)
        order = np.argsort(part, kind="stable")
        starts = np.zeros(n_parts + 1, dtype=np.int64)
        np.cumsum(np.bincount(part, minlength=n_parts), out=starts[1:])
        return ([col[lo:hi][order] for col in cols], order + lo, starts)

    chunks = list(pool.map(order_chunk, range(n_chunks)))

    def gather(p):
        pieces = [[ch[0][k][ch[2][p]:ch[2][p + 1]] for ch in chunks] for k in range(len(cols))]
        rows = np.concatenate([ch[1][ch[2][p]:ch[2][p + 1]] for ch in chunks])
        return [np.concatenate(pc) for pc in pieces], rows

    parts = list(pool.map(gather, range(n_parts)))
    return [p[0] for p in parts], [p[1] for p in parts]


def groupby(q: dict, threads: int | None = None, sort: bool = True):
    """oracle.groupby(q) over hash partitions of the rows on `threads` threads.
    Returns (keys int64[G], aggs int64[A, G]); ascending key order when
    `sort`, else partition by partition (each partition ascending)."""
    t = threads or default_threads()
    cols = [np.ascontiguousarray(c) for c in q["cols"]]
    n = len(cols[0]) if cols else 0
    if t <= 1 or n == 0:
        return _groupby(q)
    with ThreadPoolExecutor(max_workers=t) as pool:
        part_cols, _ = _split(cols, list(q["keys"]), t, pool, t)

        def run(p):
            if len(part_cols[p][0]) == 0:
                return None
            return _groupby(dict(q, cols=part_cols[p]))

        res = [r for r in pool.map(run, range(t)) if r is not None]
    n_aggs = len(q["aggs"])
    if not res:
        return np.empty(0, np.int64), np.empty((n_aggs, 0), np.int64)
    keys = np.concatenate([r[0] for r in res])
    aggs = np.concatenate([r[1] for r in res], axis=1)
    if sort:
        o = np.argsort(keys, kind="stable")
        keys, aggs = keys[o], aggs[:, o]
    return keys, aggs


def join(build_keys, payload, probe_keys, threads: int | None = None, sort: bool = True):
    """oracle.join over hash partitions of both sides on `threads` threads.
    Returns (probe_idx int32, build_idx int32, payload int64) with global row
    numbers; sorted by (probe_idx, build_idx) when `sort`."""
    t = threads or default_threads()
    bk = np.ascontiguousarray(build_keys, dtype=np.int64)
    bp = np.ascontiguousarray(payload, dtype=np.int64)
    pk = np.ascontiguousarray(probe_keys, dtype=np.int64)
    if t <= 1 or len(bk) == 0 or len(pk) == 0:
        return _join(bk, bp, pk)
    with ThreadPoolExecutor(max_workers=t) as pool:
        b_cols, b_rows = _split([bk, bp], [0], t, pool, t)
        p_cols, p_rows = _split([pk], [0], t, pool, t)

        def run(p):
            if len(b_rows[p]) == 0 or len(p_rows[p]) == 0:
                return None
            i, j, y = _join(b_cols[p][0], b_cols[p][1], p_cols[p][0])
            return p_rows[p][i].astype(np.int32), b_rows[p][j].astype(np.int32), y

        res = [r for r in pool.map(run, range(t)) if r is not None]
    if not res:
        return np.empty(0, np.int32), np.empty(0, np.int32), np.empty(0, np.int64)
    pi, bi, y = (np.concatenate([r[k] for r in res]) for k in range(3))
    if sort:
        o = np.lexsort((bi, pi))
        pi, bi, y = pi[o], bi[o], y[o]
    return pi, bi, y
