"""Seeded synthetic inputs for the relational hot path.

Input production only: nothing here hashes, aggregates or matches.  Both the
CPU oracle (``oracle/``) and the GPU path consume the arrays these functions
return, so a parity test compares the two on identical bytes.

The paper's workload is TPC-H run through a GPU query engine (Sec. 3.2); none
of that data exists here.  These generators stand in for it with columns of
the same shapes and value ranges as the fused filter + aggregate and the
equi-join the paper profiles (Sec. 7, Table 9).  Every value is a pure
function of (seed, column tag, row index) -- see ``gen.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

# column tags (one independent stream per column)
TAG_FLAG, TAG_STATUS, TAG_QTY, TAG_PRICE, TAG_DISC, TAG_TAX, TAG_DATE = range(0x11, 0x18)
TAG_KEY, TAG_VAL = 0x21, 0x22

HIT_90 = 9 * ((1 << 64) // 10)  # P(present) = 0.9 for the join probe side


def build(force: bool = False) -> str:
    """Compile gen.c into synth/_build/libsynth.so (host C, any arch)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            lib.syn_mix64.restype = u64
            lib.syn_mix64.argtypes = [u64]
            lib.syn_draw.restype = u64
            lib.syn_draw.argtypes = [u64, u64, u64]
            lib.syn_uniform_at.restype = i64
            lib.syn_uniform_at.argtypes = [u64, u64, u64, i64, i64]
            lib.syn_uniform.argtypes = [vp, i64, ctypes.c_int, i64, i64, u64, u64]
            lib.syn_uniform_mixed.argtypes = [vp, i64, i64, i64, u64, u64]
            lib.syn_perm40.restype = u64
            lib.syn_perm40.argtypes = [u64, u64]
            lib.syn_join_build.argtypes = [vp, vp, i64, u64]
            lib.syn_join_probe.argtypes = [vp, vp, i64, i64, u64, u64]
            lib.syn_zipf_new.restype = vp
            lib.syn_zipf_new.argtypes = [i64, ctypes.c_double]
            lib.syn_zipf_free.argtypes = [vp]
            lib.syn_zipf_rank_of.restype = i64
            lib.syn_zipf_rank_of.argtypes = [vp, ctypes.c_double]
            lib.syn_zipf_keys.argtypes = [vp, vp, i64, u64, u64, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def mix64(x: int) -> int:
    """One splitmix64 step (a bijection on 64-bit words)."""
    return int(_L().syn_mix64(x & (2**64 - 1)))


def mix64_signed(x: int) -> int:
    v = mix64(x)
    return v - (1 << 64) if v >= (1 << 63) else v


def uniform(n: int, lo: int, hi: int, seed: int, tag: int, dtype=np.int64) -> np.ndarray:
    """n draws of U[lo, hi] (inclusive), stored as dtype (uint8, int32 or int64)."""
    out = np.empty(n, dtype=dtype)
    if n:
        _L().syn_uniform(_ptr(out), n, out.itemsize, lo, hi, seed, tag)
    return out


def uniform_mixed(n: int, lo: int, hi: int, seed: int, tag: int) -> np.ndarray:
    """n keys mix64(U[lo, hi]): (hi - lo + 1) distinct keys spread over int64."""
    out = np.empty(n, dtype=np.int64)
    if n:
        _L().syn_uniform_mixed(_ptr(out), n, lo, hi, seed, tag)
    return out


def lineitem(n: int, seed: int = 0) -> dict:
    """Fused filter + group-by columns (a lineitem-like fact table).

    flag U{0..2} u8, status U{0..1} u8, qty U[1,50], price U[90000,10500000]
    (cents), disc U[0,10], tax U[0,8] (all int64), date U[0,2526] int32.
    """
    return {
        "flag": uniform(n, 0, 2, seed, TAG_FLAG, np.uint8),
        "status": uniform(n, 0, 1, seed, TAG_STATUS, np.uint8),
        "qty": uniform(n, 1, 50, seed, TAG_QTY),
        "price": uniform(n, 90000, 10500000, seed, TAG_PRICE),
        "disc": uniform(n, 0, 10, seed, TAG_DISC),
        "tax": uniform(n, 0, 8, seed, TAG_TAX),
        "date": uniform(n, 0, 2526, seed, TAG_DATE, np.int32),
    }


def perm40(x: int, seed: int) -> int:
    return int(_L().syn_perm40(x, seed))


def join_build(n_b: int, seed: int = 0):
    """Build side: n_b distinct keys pi(0..n_b-1) over [0, 2^40), payload U[0, 2^63)."""
    keys = np.empty(n_b, dtype=np.int64)
    pay = np.empty(n_b, dtype=np.int64)
    if n_b:
        _L().syn_join_build(_ptr(keys), _ptr(pay), n_b, seed)
    return keys, pay


def join_probe(n_p: int, n_b: int, seed: int = 0, hit_threshold: int = HIT_90):
    """Probe side: each row present with P = hit_threshold / 2^64 (a uniform
    build key), else a key guaranteed absent from the build side.

    Returns (keys int64[n_p], present uint8[n_p]).
    """
    if not (1 <= n_b < (1 << 40)):
        raise ValueError("n_b must be in [1, 2^40)")
    keys = np.empty(n_p, dtype=np.int64)
    present = np.empty(n_p, dtype=np.uint8)
    if n_p:
        _L().syn_join_probe(_ptr(keys), _ptr(present), n_p, n_b, hit_threshold, seed)
    return keys, present


class Zipf:
    """Inverse-CDF table for Zipf(s) over ranks 1..n (P(k) proportional to k^-s)."""

    def __init__(self, n: int, s: float):
        self.n, self.s = n, s
        self._h = _L().syn_zipf_new(n, s)
        if not self._h:
            raise MemoryError("zipf table")

    def rank_of(self, u: float) -> int:
        return int(_L().syn_zipf_rank_of(self._h, u))

    def keys(self, n: int, seed: int, tag: int = TAG_KEY, mix: bool = True) -> np.ndarray:
        out = np.empty(n, dtype=np.int64)
        if n:
            _L().syn_zipf_keys(self._h, _ptr(out), n, seed, tag, int(mix))
        return out

    def close(self):
        if self._h:
            _L().syn_zipf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zipf_kv(n: int, seed: int = 0, n_ranks: int = 10_000_000, s: float = 1.1):
    """Large group-by input: key = mix64(rank), rank ~ Zipf(s) over 1..n_ranks;
    value U[-1e6, 1e6]."""
    z = Zipf(n_ranks, s)
    try:
        keys = z.keys(n, seed)
    finally:
        z.close()
    vals = uniform(n, -1_000_000, 1_000_000, seed, TAG_VAL)
    return keys, vals


def few_keys_kv(n: int, n_keys: int = 4, seed: int = 0):
    """Large group-by input with n_keys distinct keys mix64(1..n_keys); value U[-1e6, 1e6]."""
    keys = uniform_mixed(n, 1, n_keys, seed, TAG_KEY)
    vals = uniform(n, -1_000_000, 1_000_000, seed, TAG_VAL)
    return keys, vals


def mlp_params(seed: int, n_in: int = 264, n_h: int = 64, n_out: int = 4) -> np.ndarray:
    """Random parameters of the planner network (float32, layout W1 b1 W2 b2
    W3 b3): weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases U(-0.1, 0.1)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((n_h, n_in), (n_h, n_h), (n_out, n_h)):
        s = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-s, s, fan_out * fan_in))
        parts.append(rng.uniform(-0.1, 0.1, fan_out))
    return np.concatenate(parts).astype(np.float32)


def mlp_features(n: int, seed: int) -> np.ndarray:
    """n rows of sketch-like features (float32 [n, 264]): 256 register values
    in [0, 1], then log2 rows in [10, 26], four shares in [0, 1], a run
    length in [1, 64] and a key width in {0.5, 1}."""
    rng = np.random.default_rng(seed)
    x = np.empty((n, 264), dtype=np.float64)
    x[:, :256] = rng.integers(0, 58, (n, 256)) / 57.0
    x[:, 256] = rng.uniform(10, 26, n)
    x[:, 257:261] = rng.uniform(0, 1, (n, 4))
    x[:, 258] = rng.uniform(0, 64, n)
    x[:, 261] = rng.uniform(0, 1, n)
    x[:, 262] = rng.uniform(1, 64, n)
    x[:, 263] = rng.choice([0.5, 1.0], n)
    return x.astype(np.float32)
