"""Thin ctypes binding over librel.so (include/rel.h).

Argument marshalling only: every step of the group-by and join runs in the
library's CUDA kernels.  torch supplies device memory (the caching allocator)
and the current stream.  There is no CPU fallback: without the compiled
library and a CUDA device every call raises.

Query descriptions are dicts:
    cols  : list of CUDA tensors (torch.uint8, torch.int32 or torch.int64), equal length
    keys  : list of column indices
    preds : list of (col, lo, hi), inclusive
    aggs  : list of (op, base_col, [(fcol, c, s), ...]); op in sum/count/min/max
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

REL_OK, REL_E_INVALID, REL_E_CAPACITY, REL_E_CUDA = 0, -1, -2, -3
REL_E_TIMEOUT, REL_E_UNSUPPORTED, REL_E_OVERFLOW = -4, -5, -6
STATUS_NAMES = {0: "REL_OK", -1: "REL_E_INVALID", -2: "REL_E_CAPACITY", -3: "REL_E_CUDA",
                -4: "REL_E_TIMEOUT", -5: "REL_E_UNSUPPORTED", -6: "REL_E_OVERFLOW"}
U8, I32, I64 = 0, 1, 2
OPS = {"sum": 0, "count": 1, "min": 2, "max": 3}
VAR_AUTO, VAR_SMEM, VAR_GLOBAL, VAR_PARTITIONED = 0, 1, 2, 3
PLAN_EXACT, PLAN_LEARNED, PLAN_GENERIC, PLAN_SKETCH = 1, 2, 4, 8
PLAN_FELL_BACK = 0x10000
PLAN_HLL_SIZED = 0x20000
PLAN_TEST_STALL = 0x40000000  # test hook: the staged kernel's ring never drains
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 264, 64, 4, 21380


def plan_force(variant: int) -> int:
    """Flag bits that force a group-by variant (VAR_SMEM / VAR_GLOBAL / VAR_PARTITIONED)."""
    return variant << 8


OP_GROUPBY, OP_JOIN_PROBE = 0, 1
MAX_COLS, MAX_KEYS, MAX_PREDS, MAX_AGGS = 8, 4, 4, 8

_DT = {torch.uint8: U8, torch.int32: I32, torch.int64: I64}


class RelError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Col(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("type", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RangePred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lo", ctypes.c_int64),
                ("hi", ctypes.c_int64)]


class Agg(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("base_col", ctypes.c_int32), ("nf", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fcol", ctypes.c_int32 * 2),
                ("c", ctypes.c_int64 * 2), ("s", ctypes.c_int64 * 2)]


class GroupByDesc(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int32),
                ("n_keys", ctypes.c_int32), ("n_preds", ctypes.c_int32),
                ("n_aggs", ctypes.c_int32), ("cols", ctypes.POINTER(Col)),
                ("key_cols", ctypes.POINTER(ctypes.c_int32)),
                ("preds", ctypes.POINTER(RangePred)), ("aggs", ctypes.POINTER(Agg))]


class Plan(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int64), ("variant", ctypes.c_int32),
                ("smem_slots", ctypes.c_int32), ("workspace_bytes", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64), ("est_groups", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("tiny_slots", ctypes.c_int32),
                ("tiny_mult", ctypes.c_uint32), ("n_hot", ctypes.c_int32),
                ("hot_keys", ctypes.c_int64 * 32), ("tile_rows", ctypes.c_int32),
                ("n_stages", ctypes.c_int32), ("part_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def __repr__(self):
        return (f"Plan(slots={self.slots}, variant={self.variant}, tiny_slots={self.tiny_slots}, "
                f"n_hot={self.n_hot}, "
                f"smem_slots={self.smem_slots}, workspace_bytes={self.workspace_bytes}, "
                f"est_groups={self.est_groups})")

    def layers(self, tiny: int, smem: int, variant: int | None = None) -> "Plan":
        """Set the per-CTA layers (thread-private slots, CTA-shared slots); drops
        any pinned hot keys."""
        self.tiny_slots, self.smem_slots = tiny, smem
        self.n_hot = 0
        if variant is not None:
            self.variant = variant
        return self


class SketchInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("sample_rows", ctypes.c_int32),
                ("kept", ctypes.c_int32), ("ndv", ctypes.c_int32),
                ("singletons", ctypes.c_int32), ("runs", ctypes.c_int32),
                ("key_bits", ctypes.c_int32), ("key_min", ctypes.c_int64),
                ("key_max", ctypes.c_int64), ("top_key", ctypes.c_int64 * 32),
                ("top_count", ctypes.c_int32 * 32), ("hll", ctypes.c_uint8 * 256),
                ("features", ctypes.c_float * 264)]


class JoinTableC(ctypes.Structure):
    _fields_ = [("ws", ctypes.c_void_p), ("slots", ctypes.c_int64), ("n_build", ctypes.c_int64),
                ("log2_slots", ctypes.c_int32), ("magic", ctypes.c_int32),
                ("reserved", ctypes.c_uint64 * 4)]


class JoinProbeDesc(ctypes.Structure):
    _fields_ = [("table", ctypes.POINTER(JoinTableC)), ("probe_keys", ctypes.c_void_p),
                ("n_probe", ctypes.c_int64)]


BATCH_MAX_AGGS = 4
REL_BATCH_MAX_AGGS_PY = BATCH_MAX_AGGS


def _np_fmt(t):
    if t in (ctypes.c_void_p, ctypes.c_uint64):
        return np.uint64
    if t is ctypes.c_int64:
        return np.int64
    if t is ctypes.c_int32:
        return np.int32
    if t is ctypes.c_uint32:
        return np.uint32
    if hasattr(t, "_length_"):
        return (_np_fmt(t._type_), (t._length_,))
    if isinstance(t, type) and issubclass(t, ctypes._Pointer):
        return np.uint64
    raise TypeError(t)


def _np_dtype(ct):
    """A numpy dtype with the exact layout of a ctypes structure."""
    names = [n for n, _ in ct._fields_]
    return np.dtype({"names": names, "formats": [_np_fmt(t) for _, t in ct._fields_],
                     "offsets": [getattr(ct, n).offset for n in names],
                     "itemsize": ctypes.sizeof(ct)})


class BatchGroupBy(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("n_rows", ctypes.c_int64),
                ("key_type", ctypes.c_int32), ("n_aggs", ctypes.c_int32),
                ("ops", ctypes.c_int32 * BATCH_MAX_AGGS), ("slots", ctypes.c_int64),
                ("est_groups", ctypes.c_int64), ("out_keys", ctypes.c_void_p),
                ("out_aggs", ctypes.c_void_p * BATCH_MAX_AGGS), ("out_capacity", ctypes.c_int64)]


class BatchJoinC(ctypes.Structure):
    _fields_ = [("build_keys", ctypes.c_void_p), ("build_payload", ctypes.c_void_p),
                ("n_build", ctypes.c_int64), ("probe_keys", ctypes.c_void_p),
                ("n_probe", ctypes.c_int64), ("out_probe_idx", ctypes.c_void_p),
                ("out_build_idx", ctypes.c_void_p), ("out_payload", ctypes.c_void_p),
                ("out_capacity", ctypes.c_int64)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("items", ctypes.c_int32),
                ("probe_width", ctypes.c_int32), ("smem_max_groups", ctypes.c_int32)]

    def astuple(self):
        return (self.block, self.items, self.probe_width, self.smem_max_groups)


class BatchHandle(ctypes.Structure):
    _fields_ = [("words", ctypes.c_uint64 * 40)]


_lock = threading.Lock()
_lib = None

# every function include/rel.h declares (the ABI test checks the header agrees)
EXPORTS = ["rel_plan_size", "rel_groupby_agg", "rel_groupby_ws_bytes", "rel_join_ws_bytes",
           "rel_join_build", "rel_join_probe", "rel_last_error", "rel_launch_count",
           "rel_version", "rel_profile_start", "rel_profile_stop", "rel_kernel_name",
           "rel_groupby_agg_static", "rel_sketch", "rel_sketch_ws_bytes", "rel_plan_ws_bytes",
           "rel_groupby_auto", "rel_groupby_auto_ws_bytes", "rel_mlp_round", "rel_mlp_forward",
           "rel_mlp_ws_bytes", "rel_mlp_backward", "rel_mlp_adamw", "rel_planner_set",
           "rel_batch_ws_bytes", "rel_batch_prepare", "rel_batch_run", "rel_batch_results",
           "rel_batch_autotune", "rel_sketch_batched", "rel_sketch_batched_ws_bytes",
           "rel_plan_learned_rule", "rel_plan_size_batched", "rel_plan_size_batched_ws_bytes",
           "rel_shard_ws_bytes", "rel_shard_split", "rel_key_hll_ws_bytes", "rel_key_hll"]
SHARD_MAX_WORLD = 64
SKETCH_TOP, SKETCH_FEATURES = 32, 264
STATIC_MAX_GROUPS = 32768


def lib_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load librel.so (building it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_stale and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"librel.so is missing ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i64, i32, u32, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint32, ctypes.c_uint64)
        L.rel_plan_size.restype = i32
        L.rel_plan_size.argtypes = [i32, vp, u32, i64, vp, ctypes.c_size_t, ctypes.POINTER(Plan), vp]
        L.rel_groupby_agg.restype = i32
        L.rel_groupby_agg.argtypes = [ctypes.POINTER(GroupByDesc), ctypes.POINTER(Plan), vp,
                                      ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_void_p), i64,
                                      ctypes.POINTER(i64), vp]
        L.rel_groupby_ws_bytes.restype = u64
        L.rel_groupby_ws_bytes.argtypes = [i64, i32]
        L.rel_join_ws_bytes.restype = u64
        L.rel_join_ws_bytes.argtypes = [i64]
        L.rel_join_build.restype = i32
        L.rel_join_build.argtypes = [vp, vp, i64, vp, ctypes.c_size_t, ctypes.POINTER(JoinTableC), vp]
        L.rel_join_probe.restype = i32
        L.rel_join_probe.argtypes = [ctypes.POINTER(JoinTableC), vp, i64, vp, vp, vp, i64,
                                     ctypes.POINTER(i64), vp]
        L.rel_last_error.restype = ctypes.c_char_p
        L.rel_last_error.argtypes = []
        L.rel_launch_count.restype = u64
        L.rel_launch_count.argtypes = []
        L.rel_version.restype = i32
        L.rel_version.argtypes = []
        L.rel_profile_start.restype = None
        L.rel_profile_start.argtypes = []
        L.rel_profile_stop.restype = i64
        L.rel_profile_stop.argtypes = [vp, vp, i64]
        L.rel_kernel_name.restype = ctypes.c_char_p
        L.rel_kernel_name.argtypes = [i32]
        L.rel_plan_ws_bytes.restype = u64
        L.rel_plan_ws_bytes.argtypes = [ctypes.POINTER(Plan), i32, i64]
        L.rel_sketch_ws_bytes.restype = u64
        L.rel_sketch_ws_bytes.argtypes = []
        L.rel_sketch.restype = i32
        L.rel_sketch.argtypes = [ctypes.POINTER(GroupByDesc), vp, ctypes.c_size_t,
                                 ctypes.POINTER(SketchInfo), vp]
        L.rel_groupby_agg_static.restype = i32
        L.rel_groupby_agg_static.argtypes = [ctypes.POINTER(GroupByDesc), i64, vp,
                                             ctypes.POINTER(ctypes.c_void_p), i64,
                                             ctypes.POINTER(i64), vp]
        L.rel_groupby_auto.restype = i32
        L.rel_groupby_auto.argtypes = [ctypes.POINTER(GroupByDesc), u32, vp, ctypes.c_size_t, vp,
                                       ctypes.POINTER(ctypes.c_void_p), i64, ctypes.POINTER(i64),
                                       ctypes.POINTER(Plan), vp]
        L.rel_groupby_auto_ws_bytes.restype = u64
        L.rel_groupby_auto_ws_bytes.argtypes = [ctypes.POINTER(GroupByDesc)]
        L.rel_mlp_round.restype = i32
        L.rel_mlp_round.argtypes = [vp, vp, vp]
        L.rel_mlp_forward.restype = i32
        L.rel_mlp_forward.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.rel_mlp_ws_bytes.restype = u64
        L.rel_mlp_ws_bytes.argtypes = [i32]
        L.rel_mlp_backward.restype = i32
        L.rel_mlp_backward.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, ctypes.c_size_t, vp, vp,
                                       vp]
        L.rel_mlp_adamw.restype = i32
        L.rel_mlp_adamw.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
        L.rel_planner_set.restype = i32
        L.rel_planner_set.argtypes = [vp, vp]
        L.rel_sketch_batched_ws_bytes.restype = u64
        L.rel_sketch_batched_ws_bytes.argtypes = [i32]
        L.rel_sketch_batched.restype = i32
        L.rel_sketch_batched.argtypes = [ctypes.POINTER(GroupByDesc), i32, vp, ctypes.c_size_t,
                                         ctypes.POINTER(SketchInfo), vp]
        L.rel_plan_learned_rule.restype = i32
        L.rel_plan_learned_rule.argtypes = [ctypes.POINTER(SketchInfo), vp, i64, i32,
                                            ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.rel_plan_size_batched_ws_bytes.restype = u64
        L.rel_plan_size_batched_ws_bytes.argtypes = [i32]
        L.rel_plan_size_batched.restype = i32
        L.rel_plan_size_batched.argtypes = [ctypes.POINTER(GroupByDesc), i32, u32, vp,
                                            ctypes.c_size_t, ctypes.POINTER(Plan), vp]
        L.rel_key_hll_ws_bytes.restype = u64
        L.rel_key_hll_ws_bytes.argtypes = []
        L.rel_key_hll.restype = i32
        L.rel_key_hll.argtypes = [vp, i32, i64, vp, ctypes.c_size_t, vp,
                                  ctypes.POINTER(ctypes.c_double), vp]
        L.rel_shard_ws_bytes.restype = u64
        L.rel_shard_ws_bytes.argtypes = [i32]
        L.rel_shard_split.restype = i32
        L.rel_shard_split.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p), i32, i64, i32, vp,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(i64), vp,
                                      ctypes.c_size_t, vp]
        PG, PJ = ctypes.POINTER(BatchGroupBy), ctypes.POINTER(BatchJoinC)
        PC, PH = ctypes.POINTER(BatchConfig), ctypes.POINTER(BatchHandle)
        L.rel_batch_ws_bytes.restype = u64
        L.rel_batch_ws_bytes.argtypes = [PG, i32, PJ, i32]
        L.rel_batch_prepare.restype = i32
        L.rel_batch_prepare.argtypes = [PG, i32, PJ, i32, PC, vp, ctypes.c_size_t, PH, vp]
        L.rel_batch_run.restype = i32
        L.rel_batch_run.argtypes = [PH, vp]
        L.rel_batch_results.restype = i32
        L.rel_batch_results.argtypes = [PH, ctypes.POINTER(i64), ctypes.POINTER(u32), vp]
        L.rel_batch_autotune.restype = i32
        L.rel_batch_autotune.argtypes = [PG, i32, PJ, i32, PC, i32, i32, vp, ctypes.c_size_t, PH,
                                         PC, ctypes.POINTER(ctypes.c_float), vp]
        _lib = L
        return L


def _check(status: int, allow=()) -> int:
    if status != REL_OK and status not in allow:
        raise RelError(status, load().rel_last_error().decode())
    return status


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def launch_count() -> int:
    return int(load().rel_launch_count())


def profile_start() -> None:
    """Record a CUDA event pair around every later library launch."""
    load().rel_profile_start()


def profile_stop():
    """Stop recording; returns [(kernel name, milliseconds), ...] in launch order."""
    L = load()
    n = L.rel_profile_stop(None, None, 0)
    if n < 0:
        raise RelError(REL_E_CUDA, "profile events")
    ids = (ctypes.c_int32 * max(1, n))()
    ms = (ctypes.c_float * max(1, n))()
    L.rel_profile_stop(ids, ms, n)
    return [(L.rel_kernel_name(ids[i]).decode(), float(ms[i])) for i in range(n)]


class _Desc:
    """Keeps the ctypes arrays of one descriptor alive."""

    def __init__(self, q: dict):
        cols = q["cols"]
        if not cols:
            raise ValueError("no columns")
        n = cols[0].numel()
        for c in cols:
            if c.dtype not in _DT or c.numel() != n or not c.is_cuda or not c.is_contiguous():
                raise ValueError("columns must be contiguous CUDA uint8/int32/int64 of one length")
        self.tensors = cols
        self.cols = (Col * len(cols))(*[Col(c.data_ptr(), _DT[c.dtype], 0) for c in cols])
        self.keys = (ctypes.c_int32 * max(1, len(q["keys"])))(*q["keys"])
        preds = q.get("preds", [])
        self.preds = (RangePred * max(1, len(preds)))(*[RangePred(c, 0, lo, hi) for c, lo, hi in preds])
        aggs = []
        for op, base, fs in q["aggs"]:
            a = Agg(OPS[op], base, len(fs), 0)
            for f, (fc, c, s) in enumerate(fs):
                a.fcol[f], a.c[f], a.s[f] = fc, c, s
            aggs.append(a)
        self.aggs = (Agg * max(1, len(aggs)))(*aggs)
        self.n_aggs = len(aggs)
        self.d = GroupByDesc(n, len(cols), len(q["keys"]), len(preds), len(aggs), self.cols,
                             self.keys, self.preds, self.aggs)


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def plan_groupby(q: dict, flags: int = 0, groups_hint: int = 0, stream=None) -> Plan:
    """rel_plan_size for a group-by (REL_PLAN_EXACT runs the GPU distinct count)."""
    L = load()
    d = _Desc(q)
    plan = Plan()
    dev = q["cols"][0].device
    st = _stream(stream)
    r = L.rel_plan_size(OP_GROUPBY, ctypes.byref(d.d), flags, groups_hint, None, 0,
                        ctypes.byref(plan), st)
    if r == REL_E_CAPACITY and plan.scratch_bytes:
        ws = _ws(plan.scratch_bytes, dev)
        r = L.rel_plan_size(OP_GROUPBY, ctypes.byref(d.d), flags, groups_hint, ws.data_ptr(),
                            ws.numel(), ctypes.byref(plan), st)
    _check(r)
    return plan


def groupby(q: dict, plan: Plan | None = None, flags: int = 0, groups_hint: int = 0,
            capacity: int | None = None, ws: torch.Tensor | None = None, stream=None):
    """Run the fused filter + group-by.  Returns (keys int64[G], [agg int64[G], ...])
    in unspecified group order."""
    L = load()
    d = _Desc(q)
    dev = q["cols"][0].device
    if plan is None:
        plan = plan_groupby(q, flags=flags, groups_hint=groups_hint, stream=stream)
    if capacity is None:
        capacity = max(1, plan.est_groups + 1)
    need = int(L.rel_plan_ws_bytes(ctypes.byref(plan), d.n_aggs, d.d.n_rows))
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    st = _stream(stream)
    while True:
        keys = torch.empty(capacity, dtype=torch.int64, device=dev)
        aggs = [torch.empty(capacity, dtype=torch.int64, device=dev) for _ in range(d.n_aggs)]
        ptrs = (ctypes.c_void_p * max(1, d.n_aggs))(*[a.data_ptr() for a in aggs])
        n = ctypes.c_int64(0)
        r = L.rel_groupby_agg(ctypes.byref(d.d), ctypes.byref(plan), ws.data_ptr(), ws.numel(),
                              keys.data_ptr(), ptrs, capacity, ctypes.byref(n), st)
        if r == REL_E_CAPACITY and n.value > capacity:
            capacity = n.value
            continue
        _check(r)
        g = n.value
        return keys[:g], [a[:g] for a in aggs]


def groupby_static(q: dict, max_groups: int, capacity: int | None = None, stream=None):
    """Group-by through rel_groupby_agg_static: the library allocates nothing
    (its hash table is a scratch array built into librel.so), for callers
    that cannot allocate device memory.  The outputs here are allocated by
    the caller (this function), as the C entry point requires.  Returns
    (keys int64[G], [agg int64[G], ...]) in unspecified group order."""
    L = load()
    d = _Desc(q)
    dev = q["cols"][0].device
    cap = max(1, capacity if capacity is not None else max_groups)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    aggs = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(d.n_aggs)]
    ptrs = (ctypes.c_void_p * max(1, d.n_aggs))(*[a.data_ptr() for a in aggs])
    n = ctypes.c_int64(0)
    _check(L.rel_groupby_agg_static(ctypes.byref(d.d), max_groups, keys.data_ptr(), ptrs, cap,
                                    ctypes.byref(n), _stream(stream)))
    g = n.value
    return keys[:g], [a[:g] for a in aggs]


def groupby_auto(q: dict, flags: int = 0, capacity: int | None = None,
                 ws: torch.Tensor | None = None, stream=None):
    """rel_groupby_auto: plan (flags as plan_groupby) and run in one call; an
    overflowing learned plan is re-planned exactly.  Returns (keys, aggs, plan).
    Default output capacity: one row per input row (always sufficient)."""
    L = load()
    d = _Desc(q)
    dev = q["cols"][0].device
    need = int(L.rel_groupby_auto_ws_bytes(ctypes.byref(d.d)))
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    cap = max(1, d.d.n_rows if capacity is None else capacity)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    aggs = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(d.n_aggs)]
    ptrs = (ctypes.c_void_p * max(1, d.n_aggs))(*[a.data_ptr() for a in aggs])
    n = ctypes.c_int64(0)
    plan = Plan()
    _check(L.rel_groupby_auto(ctypes.byref(d.d), flags, ws.data_ptr(), ws.numel(),
                              keys.data_ptr(), ptrs, cap, ctypes.byref(n), ctypes.byref(plan),
                              _stream(stream)))
    g = n.value
    return keys[:g], [a[:g] for a in aggs], plan


def auto_ws_bytes(q: dict) -> int:
    return int(load().rel_groupby_auto_ws_bytes(ctypes.byref(_Desc(q).d)))


def key_hll(keys: torch.Tensor, stream=None):
    """rel_key_hll: (registers uint32[4096] as numpy, estimate) of a key column."""
    L = load()
    if keys.dtype not in (torch.int32, torch.int64) or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA int32 / int64 tensor")
    ws = _ws(L.rel_key_hll_ws_bytes(), keys.device)
    regs = np.zeros(4096, dtype=np.uint32)
    est = ctypes.c_double()
    _check(L.rel_key_hll(keys.data_ptr(), _DT[keys.dtype], keys.numel(), ws.data_ptr(), ws.numel(),
                         regs.ctypes.data, ctypes.byref(est), _stream(stream)))
    return regs, est.value


def shard_split(keys: torch.Tensor, words: list, world: int, stream=None):
    """rel_shard_split: the groups (keys, words) regrouped by owner rank.
    Returns (keys, [words], counts per owner)."""
    L = load()
    n = keys.numel()
    for t in [keys, *words]:
        if t.dtype != torch.int64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError("keys and words must be contiguous CUDA int64 tensors of one length")
    dev = keys.device
    out_k = torch.empty(max(1, n), dtype=torch.int64, device=dev)[:n]
    out_w = [torch.empty(max(1, n), dtype=torch.int64, device=dev)[:n] for _ in words]
    nw = len(words)
    wp = (ctypes.c_void_p * max(1, nw))(*[w.data_ptr() for w in words])
    op = (ctypes.c_void_p * max(1, nw))(*[w.data_ptr() for w in out_w])
    counts = (ctypes.c_int64 * max(1, world))()
    ws = _ws(L.rel_shard_ws_bytes(world), dev)
    _check(L.rel_shard_split(keys.data_ptr(), wp, nw, n, world, out_k.data_ptr(), op, counts,
                             ws.data_ptr(), ws.numel(), _stream(stream)))
    return out_k, out_w, [int(counts[r]) for r in range(world)]


# ---------------------------------------------------------- planner network

def _f32(t: torch.Tensor, n: int | None = None) -> int:
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32 tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"expected at least {n} elements")
    return t.data_ptr()


def mlp_round(params: torch.Tensor, bf16: torch.Tensor, stream=None) -> None:
    """bf16 <- round-to-nearest-even(params) (rel_mlp_round)."""
    if bf16.dtype != torch.bfloat16 or bf16.numel() < MLP_PARAMS:
        raise ValueError("bf16 must hold MLP_PARAMS bfloat16 values")
    _check(load().rel_mlp_round(_f32(params, MLP_PARAMS), bf16.data_ptr(), _stream(stream)))


def mlp_forward(bf16: torch.Tensor, params: torch.Tensor, x: torch.Tensor,
                acts: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y[B, 4] for x[B, 264] (rel_mlp_forward); acts[B, 128] receives the
    hidden pre-activations when given."""
    B = x.shape[0]
    out = torch.empty((B, MLP_OUT), dtype=torch.float32, device=x.device)
    _check(load().rel_mlp_forward(bf16.data_ptr(), _f32(params, MLP_PARAMS), _f32(x, B * MLP_IN),
                                  B, out.data_ptr(),
                                  None if acts is None else _f32(acts, B * 2 * MLP_HIDDEN),
                                  _stream(stream)))
    return out


def mlp_backward(bf16: torch.Tensor, x: torch.Tensor, acts: torch.Tensor, out: torch.Tensor,
                 t_ndv: torch.Tensor, t_var: torch.Tensor, grad: torch.Tensor,
                 loss: torch.Tensor, ws: torch.Tensor | None = None, stream=None) -> None:
    """grad <- d(batch-mean loss)/d(params), loss[0] <- the loss (rel_mlp_backward)."""
    L = load()
    B = x.shape[0]
    need = int(L.rel_mlp_ws_bytes(B))
    if ws is None or ws.numel() < need:
        ws = _ws(need, x.device)
    if t_var.dtype != torch.int32 or not t_var.is_contiguous() or t_var.numel() < B:
        raise ValueError("t_var must be contiguous int32[B]")
    _check(L.rel_mlp_backward(bf16.data_ptr(), _f32(x, B * MLP_IN), _f32(acts, B * 2 * MLP_HIDDEN),
                              _f32(out, B * MLP_OUT), _f32(t_ndv, B), t_var.data_ptr(), B,
                              ws.data_ptr(), ws.numel(), _f32(grad, MLP_PARAMS), _f32(loss, 1),
                              _stream(stream)))


def mlp_adamw(params: torch.Tensor, bf16: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
              grad: torch.Tensor, step: int, lr: float = 1e-3, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, weight_decay: float = 1e-4,
              stream=None) -> None:
    """One AdamW step on the parameters, refreshing the BF16 copy (rel_mlp_adamw)."""
    _check(load().rel_mlp_adamw(_f32(params, MLP_PARAMS), bf16.data_ptr(), _f32(m, MLP_PARAMS),
                                _f32(v, MLP_PARAMS), _f32(grad, MLP_PARAMS), step, lr, beta1,
                                beta2, eps, weight_decay, _stream(stream)))


_planner_ref = None  # keeps the registered parameter tensors alive


def planner_set(params: torch.Tensor | None) -> None:
    """Register FP32 parameters (and a BF16 copy made here) as the network
    REL_PLAN_LEARNED consults; None clears."""
    global _planner_ref
    L = load()
    if params is None:
        _check(L.rel_planner_set(None, None))
        _planner_ref = None
        return
    p = params.detach().to(torch.float32).contiguous()
    bf = torch.empty(MLP_PARAMS, dtype=torch.bfloat16, device=p.device)
    mlp_round(p, bf)
    torch.cuda.current_stream(p.device).synchronize()
    _check(L.rel_planner_set(bf.data_ptr(), _f32(p, MLP_PARAMS)))
    _planner_ref = (p, bf)


def sketch(q: dict, stream=None) -> "SketchInfo":
    """rel_sketch: the 4096-row sample summary of a group-by input."""
    L = load()
    d = _Desc(q)
    ws = _ws(L.rel_sketch_ws_bytes(), q["cols"][0].device)
    out = SketchInfo()
    _check(L.rel_sketch(ctypes.byref(d.d), ws.data_ptr(), ws.numel(), ctypes.byref(out),
                        _stream(stream)))
    return out


def sketch_batched(qs: list, stream=None) -> list:
    """rel_sketch_batched: the sample summaries of many inputs, one launch."""
    L = load()
    if not qs:
        return []
    ds = [_Desc(q) for q in qs]
    arr = (GroupByDesc * len(ds))(*[d.d for d in ds])
    ws = _ws(L.rel_sketch_batched_ws_bytes(len(ds)), qs[0]["cols"][0].device)
    out = (SketchInfo * len(ds))()
    _check(L.rel_sketch_batched(arr, len(ds), ws.data_ptr(), ws.numel(), out, _stream(stream)))
    return list(out)


def _kv_descs(keys: list, vals: list, ops):
    """Key/value descriptors (one int32/int64 key column, one int64 value
    column) built column-wise; returns (ctypes array, objects to keep alive)."""
    n = len(keys)
    cols = np.zeros(2 * n, dtype=_np_dtype(Col))
    cols["data"][0::2] = [k.data_ptr() for k in keys]
    cols["type"][0::2] = [_DT[k.dtype] for k in keys]
    cols["data"][1::2] = [v.data_ptr() for v in vals]
    cols["type"][1::2] = I64
    kc = np.zeros(1, dtype=np.int32)
    aggs = (Agg * len(ops))(*[Agg(OPS[op], 1, 0, 0) for op in ops])
    d = np.zeros(n, dtype=_np_dtype(GroupByDesc))
    d["n_rows"] = [k.numel() for k in keys]
    d["n_cols"], d["n_keys"], d["n_preds"], d["n_aggs"] = 2, 1, 0, len(ops)
    d["cols"] = cols.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(2 * ctypes.sizeof(Col))
    d["key_cols"] = kc.ctypes.data
    d["preds"] = 0
    d["aggs"] = ctypes.addressof(aggs)
    arr = (GroupByDesc * n).from_buffer(d)
    return arr, (cols, kc, aggs, d)


def sketch_kv_batched(keys: list, vals: list, ops=("sum", "count"), stream=None) -> list:
    """sketch_batched for key/value inputs (one int32/int64 key column, one
    int64 value column), descriptors built column-wise."""
    L = load()
    n = len(keys)
    if n == 0:
        return []
    arr, keep = _kv_descs(keys, vals, ops)
    ws = _ws(L.rel_sketch_batched_ws_bytes(n), keys[0].device)
    out = (SketchInfo * n)()
    _check(L.rel_sketch_batched(arr, n, ws.data_ptr(), ws.numel(), out, _stream(stream)))
    return list(out)


def plan_kv_batched(keys: list, vals: list, ops=("sum", "count"), flags: int = PLAN_LEARNED,
                    stream=None) -> list:
    """rel_plan_size_batched for key/value inputs: learned plans of all of
    them from one sketch launch and one network launch (the registered
    network)."""
    L = load()
    n = len(keys)
    if n == 0:
        return []
    arr, keep = _kv_descs(keys, vals, ops)
    ws = _ws(L.rel_plan_size_batched_ws_bytes(n), keys[0].device)
    plans = (Plan * n)()
    _check(L.rel_plan_size_batched(arr, n, flags, ws.data_ptr(), ws.numel(), plans,
                                   _stream(stream)))
    return list(plans)


def plan_learned_rule(info: "SketchInfo", y, n_rows: int, partitioned_ok: bool = True):
    """rel_plan_learned_rule (host only): (est_groups, variant) from a sketch
    and the network's 4 outputs."""
    L = load()
    yy = np.ascontiguousarray(np.asarray(y, dtype=np.float32)[:MLP_OUT])
    est, var = ctypes.c_int64(), ctypes.c_int32()
    _check(L.rel_plan_learned_rule(ctypes.byref(info), yy.ctypes.data, n_rows,
                                   1 if partitioned_ok else 0, ctypes.byref(est),
                                   ctypes.byref(var)))
    return est.value, var.value


class JoinTable:
    """A built join table; owns its workspace tensor."""

    def __init__(self, keys: torch.Tensor, payload: torch.Tensor, stream=None):
        L = load()
        if keys.dtype != torch.int64 or payload.dtype != torch.int64 or keys.numel() != payload.numel():
            raise ValueError("build keys and payload must be int64 of one length")
        self.keys, self.payload = keys, payload
        self.ws = _ws(L.rel_join_ws_bytes(keys.numel()), keys.device)
        self.t = JoinTableC()
        _check(L.rel_join_build(keys.data_ptr(), payload.data_ptr(), keys.numel(),
                                self.ws.data_ptr(), self.ws.numel(), ctypes.byref(self.t),
                                _stream(stream)))

    def count(self, probe: torch.Tensor, stream=None) -> int:
        L = load()
        pd = JoinProbeDesc(ctypes.pointer(self.t), probe.data_ptr(), probe.numel())
        plan = Plan()
        _check(L.rel_plan_size(OP_JOIN_PROBE, ctypes.byref(pd), 0, 0, None, 0,
                               ctypes.byref(plan), _stream(stream)))
        return int(plan.est_groups)

    def probe(self, probe: torch.Tensor, capacity: int | None = None, stream=None):
        """Returns (probe_idx int32, build_idx int32, payload int64), unspecified order."""
        L = load()
        if probe.dtype != torch.int64:
            raise ValueError("probe keys must be int64")
        if capacity is None:
            capacity = max(1, probe.numel())
        dev = probe.device
        while True:
            pi = torch.empty(capacity, dtype=torch.int32, device=dev)
            bi = torch.empty(capacity, dtype=torch.int32, device=dev)
            pay = torch.empty(capacity, dtype=torch.int64, device=dev)
            n = ctypes.c_int64(0)
            r = L.rel_join_probe(ctypes.byref(self.t), probe.data_ptr(), probe.numel(),
                                 pi.data_ptr(), bi.data_ptr(), pay.data_ptr(), capacity,
                                 ctypes.byref(n), _stream(stream))
            if r == REL_E_CAPACITY and n.value > capacity:
                capacity = n.value
                continue
            _check(r)
            return pi[:n.value], bi[:n.value], pay[:n.value]


# ------------------------------------------------------- batched execution

DEFAULT_BATCH_CONFIG = (256, 8, 1, 512)
# the tuner's search space: block x items x probe width x shared-memory placement
BATCH_SEARCH = [(b, it, w, sm) for b in (128, 256, 512) for it in (4, 8, 16)
                for w in (1, 2, 4, 8) for sm in (0, 512, 2048)]


class Batch:
    """Many key/value group-bys and join partitions run as one batch
    (rel_batch_*): two persistent launches, replayable from a CUDA graph.

    groupbys: dicts with keys (int32/int64 CUDA tensor), vals (int64 or None),
      ops (list of "sum"/"count"/"min"/"max"), slots (power of two), est_groups,
      capacity (output rows).
    joins: dicts with build_keys, build_payload, probe_keys (int64), capacity.
    Outputs are allocated here; inputs must stay alive and in place."""

    def __init__(self, groupbys, joins, device=None, stream=None):
        L = load()
        self.gspec, self.jspec = list(groupbys), list(joins)
        dev = device or (self.gspec[0]["keys"].device if self.gspec
                         else self.jspec[0]["build_keys"].device if self.jspec else "cuda")
        self.device = torch.device(dev)
        ng, nj = len(self.gspec), len(self.jspec)
        # descriptors in numpy structured arrays laid out as the C structs
        # (filled column-wise), outputs in a few flat tensors
        g = np.zeros(max(1, ng), dtype=_np_dtype(BatchGroupBy))
        j = np.zeros(max(1, nj), dtype=_np_dtype(BatchJoinC))
        gcap = np.array([max(1, int(q["capacity"])) for q in self.gspec], dtype=np.int64)
        gna = np.array([len(q["ops"]) for q in self.gspec], dtype=np.int64)
        self.gk_off = np.concatenate([[0], np.cumsum(gcap)]).astype(np.int64)
        self.ga_off = np.concatenate([[0], np.cumsum(gcap * gna)]).astype(np.int64)
        self.gkeys = torch.empty(max(1, int(self.gk_off[-1])), dtype=torch.int64, device=self.device)
        self.gaggs = torch.empty(max(1, int(self.ga_off[-1])), dtype=torch.int64, device=self.device)
        if ng:
            for q in self.gspec:
                k, v = q["keys"], q.get("vals")
                if k.dtype not in (torch.int32, torch.int64) or not k.is_contiguous():
                    raise ValueError("group-by keys must be contiguous int32/int64")
                if v is not None and (v.dtype != torch.int64 or v.numel() != k.numel()):
                    raise ValueError("group-by values must be int64 of the keys' length")
            g["keys"][:ng] = [q["keys"].data_ptr() for q in self.gspec]
            g["vals"][:ng] = [q["vals"].data_ptr() if q.get("vals") is not None else 0
                              for q in self.gspec]
            g["n_rows"][:ng] = [q["keys"].numel() for q in self.gspec]
            g["key_type"][:ng] = [_DT[q["keys"].dtype] for q in self.gspec]
            g["n_aggs"][:ng] = gna
            for i, q in enumerate(self.gspec):
                g["ops"][i, :len(q["ops"])] = [OPS[op] for op in q["ops"]]
            g["slots"][:ng] = [int(q["slots"]) for q in self.gspec]
            g["est_groups"][:ng] = [int(q.get("est_groups", 0)) for q in self.gspec]
            g["out_keys"][:ng] = self.gkeys.data_ptr() + 8 * self.gk_off[:-1]
            base = self.gaggs.data_ptr() + 8 * self.ga_off[:-1]
            for a in range(REL_BATCH_MAX_AGGS_PY):
                g["out_aggs"][:ng, a] = np.where(gna > a, base + 8 * a * gcap, 0)
            g["out_capacity"][:ng] = gcap
        jcap = np.array([max(1, int(q["capacity"])) for q in self.jspec], dtype=np.int64)
        self.j_off = np.concatenate([[0], np.cumsum(jcap)]).astype(np.int64)
        tot = max(1, int(self.j_off[-1]))
        self.jpi = torch.empty(tot, dtype=torch.int32, device=self.device)
        self.jbi = torch.empty(tot, dtype=torch.int32, device=self.device)
        self.jpay = torch.empty(tot, dtype=torch.int64, device=self.device)
        if nj:
            for q in self.jspec:
                for t in (q["build_keys"], q["build_payload"], q["probe_keys"]):
                    if t.dtype != torch.int64 or not t.is_contiguous():
                        raise ValueError("join columns must be contiguous int64")
            j["build_keys"][:nj] = [q["build_keys"].data_ptr() for q in self.jspec]
            j["build_payload"][:nj] = [q["build_payload"].data_ptr() for q in self.jspec]
            j["n_build"][:nj] = [q["build_keys"].numel() for q in self.jspec]
            j["probe_keys"][:nj] = [q["probe_keys"].data_ptr() for q in self.jspec]
            j["n_probe"][:nj] = [q["probe_keys"].numel() for q in self.jspec]
            j["out_probe_idx"][:nj] = self.jpi.data_ptr() + 4 * self.j_off[:-1]
            j["out_build_idx"][:nj] = self.jbi.data_ptr() + 4 * self.j_off[:-1]
            j["out_payload"][:nj] = self.jpay.data_ptr() + 8 * self.j_off[:-1]
            j["out_capacity"][:nj] = jcap
        self._gnp, self._jnp = g, j
        self.g = (BatchGroupBy * len(g)).from_buffer(g)
        self.j = (BatchJoinC * len(j)).from_buffer(j)
        need = int(L.rel_batch_ws_bytes(self.g, ng, self.j, nj))
        if need == 0 and (ng or nj):
            raise RelError(REL_E_INVALID, "invalid batch")
        self.ws = _ws(need, self.device)
        self.h = BatchHandle()
        self.config = None

    def prepare(self, config=DEFAULT_BATCH_CONFIG, stream=None):
        c = BatchConfig(*config)
        _check(load().rel_batch_prepare(self.g, len(self.gspec), self.j, len(self.jspec),
                                        ctypes.byref(c), self.ws.data_ptr(), self.ws.numel(),
                                        ctypes.byref(self.h), _stream(stream)))
        self.config = tuple(config)
        return self

    def autotune(self, candidates=None, reps: int = 3, stream=None):
        """Time every candidate (block, items, probe width, smem_max_groups);
        keeps the fastest prepared.  Returns (best, {config: ms})."""
        cands = list(candidates or BATCH_SEARCH)
        arr = (BatchConfig * len(cands))(*[BatchConfig(*c) for c in cands])
        best = BatchConfig()
        ms = (ctypes.c_float * len(cands))()
        _check(load().rel_batch_autotune(self.g, len(self.gspec), self.j, len(self.jspec), arr,
                                         len(cands), reps, self.ws.data_ptr(), self.ws.numel(),
                                         ctypes.byref(self.h), ctypes.byref(best), ms,
                                         _stream(stream)))
        self.config = best.astuple()
        return self.config, {c: float(ms[i]) for i, c in enumerate(cands)}

    def run(self, stream=None):
        _check(load().rel_batch_run(ctypes.byref(self.h), _stream(stream)))

    def capture(self):
        """A CUDA graph of one run (prepare first); replay() reruns the batch."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run(stream=s)  # warm-up outside the graph
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def results(self, stream=None):
        """(counts int64[n_g + n_j], flags uint32[n_g + n_j]); flag bit 0 =
        table overflow, bit 1 = output capacity exceeded."""
        n = len(self.gspec) + len(self.jspec)
        cnt = (ctypes.c_int64 * max(1, n))()
        fl = (ctypes.c_uint32 * max(1, n))()
        _check(load().rel_batch_results(ctypes.byref(self.h), cnt, fl, _stream(stream)))
        return [int(cnt[i]) for i in range(n)], [int(fl[i]) for i in range(n)]

    def groupby_output(self, i: int, n: int):
        k0, k1 = int(self.gk_off[i]), int(self.gk_off[i + 1])
        cap = k1 - k0
        n = min(n, cap)
        a0 = int(self.ga_off[i])
        na = len(self.gspec[i]["ops"])
        return (self.gkeys[k0:k0 + n],
                [self.gaggs[a0 + a * cap:a0 + a * cap + n] for a in range(na)])

    def join_output(self, i: int, n: int):
        o0, o1 = int(self.j_off[i]), int(self.j_off[i + 1])
        n = min(n, o1 - o0)
        return self.jpi[o0:o0 + n], self.jbi[o0:o0 + n], self.jpay[o0:o0 + n]
