"""ORACLE -- test infrastructure, not the product.

Python access to the plain single-threaded CPU definitions in ``oracle.cpp``
(filtered group-by with exact int64 aggregates; inner equi-join with payload
gather).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It imports nothing from the
GPU library and the GPU library imports nothing from it.

Query descriptions are plain dicts:
    cols  : list of numpy arrays (uint8, int32 or int64)
    keys  : list of column indices (one column, or several packed, see oracle.cpp)
    preds : list of (col, lo, hi), inclusive range filters
    aggs  : list of (op, base_col, [(fcol, c, s), ...]) with op in
            {"sum", "count", "min", "max"}; the aggregate input of row i is
            base[i] * prod (c + s * fcol[i]) mod 2^64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"sum": 0, "count": 1, "min": 2, "max": 3}
_TYPES = {np.dtype(np.uint8): 0, np.dtype(np.int32): 1, np.dtype(np.int64): 2}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.orc_free.argtypes = [vp]
            lib.orc_groupby.restype = i64
            lib.orc_groupby.argtypes = [i64, vp, vp, i32, vp, i32, vp, vp, vp, i32, vp, vp, vp,
                                        vp, vp, vp, vp, vp]
            lib.orc_join.restype = i64
            lib.orc_join.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp]
            lib.orc_join_count.restype = i64
            lib.orc_join_count.argtypes = [vp, i64, vp, i64]
            lib.orc_sketch.restype = None
            lib.orc_sketch.argtypes = [i64, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp,
                                       vp]
            _lib = lib
    return _lib


def _arr(values, dtype):
    a = np.ascontiguousarray(np.asarray(values, dtype=dtype))
    return a if a.size else np.zeros(1, dtype=dtype)


def _take(ptr, n, dtype):
    """Copy n elements from a malloc'ed oracle buffer and release it."""
    lib = _L()
    try:
        if n == 0:
            return np.empty(0, dtype=dtype)
        ct = np.ctypeslib.as_ctypes_type(np.dtype(dtype))
        buf = ctypes.cast(ptr, ctypes.POINTER(ct * n)).contents
        return np.frombuffer(buf, dtype=dtype).copy()
    finally:
        lib.orc_free(ptr)


def groupby(q: dict):
    """Filtered group-by.  Returns (keys int64[G], aggs int64[A, G]) with groups
    in ascending signed key order."""
    cols = [np.ascontiguousarray(c) for c in q["cols"]]
    n = len(cols[0]) if cols else 0
    for c in cols:
        if c.dtype not in _TYPES or len(c) != n:
            raise ValueError("columns must be uint8/int32/int64 of equal length")
    ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
    types = _arr([_TYPES[c.dtype] for c in cols], np.int32)
    keys = _arr(q["keys"], np.int32)
    preds = q.get("preds", [])
    pc = _arr([p[0] for p in preds], np.int32)
    plo = _arr([p[1] for p in preds], np.int64)
    phi = _arr([p[2] for p in preds], np.int64)
    aggs = q["aggs"]
    A = len(aggs)
    op = _arr([OPS[a[0]] for a in aggs], np.int32)
    base = _arr([a[1] for a in aggs], np.int32)
    nf = _arr([len(a[2]) for a in aggs], np.int32)
    fcol = np.zeros(2 * max(A, 1), np.int32)
    cc = np.zeros(2 * max(A, 1), np.int64)
    ss = np.zeros(2 * max(A, 1), np.int64)
    for a, (_, _, fs) in enumerate(aggs):
        if len(fs) > 2:
            raise ValueError("at most two factors per aggregate")
        for f, (fc, c, s) in enumerate(fs):
            fcol[2 * a + f], cc[2 * a + f], ss[2 * a + f] = fc, c, s
    ok_p, oa_p = ctypes.c_void_p(), ctypes.c_void_p()
    ng = _L().orc_groupby(n, ptrs, types.ctypes.data, len(q["keys"]), keys.ctypes.data,
                          len(preds), pc.ctypes.data, plo.ctypes.data, phi.ctypes.data, A,
                          op.ctypes.data, base.ctypes.data, nf.ctypes.data, fcol.ctypes.data,
                          cc.ctypes.data, ss.ctypes.data, ctypes.byref(ok_p),
                          ctypes.byref(oa_p))
    if ng < 0:
        raise MemoryError("oracle group-by")
    out_keys = _take(ok_p.value, ng, np.int64)
    out_aggs = _take(oa_p.value, ng * A, np.int64).reshape(A, ng)
    return out_keys, out_aggs


def sketch(q: dict) -> dict:
    """Sample summary (see orc_sketch) plus the 264 planner features computed
    here in double precision from the integer summary."""
    import math

    cols = [np.ascontiguousarray(c) for c in q["cols"]]
    n = len(cols[0])
    ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
    types = _arr([_TYPES[c.dtype] for c in cols], np.int32)
    keys = _arr(q["keys"], np.int32)
    preds = q.get("preds", [])
    pc = _arr([p[0] for p in preds], np.int32)
    plo = _arr([p[1] for p in preds], np.int64)
    phi = _arr([p[2] for p in preds], np.int64)
    ints = np.zeros(5, np.int32)
    mm = np.zeros(2, np.int64)
    tk = np.zeros(32, np.int64)
    tc = np.zeros(32, np.int32)
    hll = np.zeros(256, np.uint8)
    _L().orc_sketch(n, ptrs, types.ctypes.data, len(q["keys"]), keys.ctypes.data, len(preds),
                    pc.ctypes.data, plo.ctypes.data, phi.ctypes.data, ints.ctypes.data,
                    mm.ctypes.data, tk.ctypes.data, tc.ctypes.data, hll.ctypes.data)
    s = dict(zip(["sample_rows", "kept", "ndv", "singletons", "runs"], ints.tolist()))
    s.update(key_min=int(mm[0]), key_max=int(mm[1]), top_key=tk, top_count=tc, hll=hll)
    bits = {np.dtype(np.uint8): 8, np.dtype(np.int32): 32, np.dtype(np.int64): 64}
    s["key_bits"] = sum(bits[cols[k].dtype] for k in q["keys"])
    kept, ndv = s["kept"], s["ndv"]
    span = (s["key_max"] - s["key_min"]) % (1 << 64)
    stats = [
        math.log2(max(n, 1)),
        ndv / kept if kept else 0.0,
        math.log2(float(span) + 1.0) if kept else 0.0,
        int(tc[0]) / kept if kept else 0.0,
        int(tc[:8].sum()) / kept if kept else 0.0,
        s["singletons"] / ndv if ndv else 0.0,
        kept / s["runs"] if s["runs"] else 0.0,
        s["key_bits"] / 64.0,
    ]
    s["features"] = np.array([h / 57.0 for h in hll.tolist()] + stats, dtype=np.float64)
    return s


def hll_estimate(registers) -> float:
    """HyperLogLog cardinality estimate with the small-range (linear counting)
    correction of Flajolet et al. (2007), m = number of registers."""
    import math

    r = np.asarray(registers, dtype=np.float64)
    m = len(r)
    alpha = 0.7213 / (1 + 1.079 / m)
    e = alpha * m * m / np.sum(2.0 ** (-r))
    zeros = int((r == 0).sum())
    if e <= 2.5 * m and zeros:
        e = m * math.log(m / zeros)
    return float(e)


_U64 = np.uint64


def _fmix64(k: np.ndarray) -> np.ndarray:
    """MurmurHash3's 64-bit finalizer (Appleby), on uint64 arrays (wrapping)."""
    k = k.copy()
    k ^= k >> _U64(33)
    k *= _U64(0xFF51AFD7ED558CCD)
    k ^= k >> _U64(33)
    k *= _U64(0xC4CEB9FE1A85EC53)
    k ^= k >> _U64(33)
    return k


def _clz64(x: np.ndarray) -> np.ndarray:
    """Leading zero bits of each uint64 (64 for zero), by halving."""
    x = x.copy()
    n = np.zeros(x.shape, np.int64)
    for s in (32, 16, 8, 4, 2, 1):
        top = x >> _U64(64 - s)
        z = top == 0
        n += np.where(z, s, 0)
        x = np.where(z, x << _U64(s), x)
    n += (x == 0).astype(np.int64)  # x was zero throughout
    return n


def key_hll(keys, p: int = 12):
    """HyperLogLog registers (2^p) of every key of one int32 / int64 column and
    their estimate (Flajolet, Fusy, Gandouet & Meunier 2007, with the
    small-range correction): h = fmix64(key ^ 2^63) over the key's 64-bit
    two's-complement bits, register = top p bits of h, value = leading zeros
    of the remaining 64 - p bits + 1 (65 - p when they are all zero)."""
    k = np.asarray(keys).astype(np.int64).view(np.uint64) ^ _U64(1 << 63)
    h = _fmix64(k)
    idx = (h >> _U64(64 - p)).astype(np.int64)
    rest = h << _U64(p)
    rank = np.where(rest == 0, 65 - p, _clz64(rest) + 1)
    regs = np.zeros(1 << p, np.uint32)
    np.maximum.at(regs, idx, rank.astype(np.uint32))
    return regs, hll_estimate(regs)


def join(build_keys, payload, probe_keys):
    """Inner equi-join bag.  Returns (probe_idx int32, build_idx int32,
    payload int64) sorted by (probe_idx, build_idx)."""
    bk = np.ascontiguousarray(build_keys, dtype=np.int64)
    bp = np.ascontiguousarray(payload, dtype=np.int64)
    pk = np.ascontiguousarray(probe_keys, dtype=np.int64)
    a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    n = _L().orc_join(bk.ctypes.data, bp.ctypes.data, len(bk), pk.ctypes.data, len(pk),
                      ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if n < 0:
        raise MemoryError("oracle join")
    return _take(a.value, n, np.int32), _take(b.value, n, np.int32), _take(c.value, n, np.int64)


def join_count(build_keys, probe_keys) -> int:
    bk = np.ascontiguousarray(build_keys, dtype=np.int64)
    pk = np.ascontiguousarray(probe_keys, dtype=np.int64)
    return int(_L().orc_join_count(bk.ctypes.data, len(bk), pk.ctypes.data, len(pk)))


# query descriptions of the benchmark workloads (shared with the GPU side)
from synth.queries import kv_query, lineitem_query  # noqa: E402,F401
