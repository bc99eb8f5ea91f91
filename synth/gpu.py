"""GPU-generated key/value columns and the instance recipe of the planner
workload (many group-by instances of mixed size and key distribution).

Input production only (see ``gen_gpu.cu``).  The recipe of one instance is a
pure function of its seed: rows log-uniform in [rows_lo, rows_hi], a key
family drawn from uniform / Zipf(0.5) / Zipf(1.0) / Zipf(1.5) / clustered, a
key domain log-uniform in [dom_lo, dom_hi]; values U[-10^6, 10^6].
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

from . import _L as _host_lib

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_gpu.cu")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynthgpu.so")
_lock = threading.Lock()
_lib = None

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
TAG_INST = 0x31

# (name, family id, Zipf exponent)
FAMILIES = [("uniform", 0, 0.0), ("zipf0.5", 1, 0.5), ("zipf1.0", 1, 1.0), ("zipf1.5", 1, 1.5),
            ("clustered", 2, 0.0)]


def build(force: bool = False) -> str:
    """Compile gen_gpu.cu into synth/_build/libsynthgpu.so (sm_103a)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lcudart_static"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.syn_gpu_kv.restype = ctypes.c_int
            lib.syn_gpu_kv.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
            lib.syn_gpu_join_build.restype = ctypes.c_int
            lib.syn_gpu_join_build.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
            lib.syn_gpu_join_probe.restype = ctypes.c_int
            lib.syn_gpu_join_probe.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def kv(family: int, s: float, n: int, domain: int, seed: int, device="cuda", stream=None):
    """(keys int64[n], vals int64[n]) CUDA tensors of one key family."""
    import torch

    keys = torch.empty(max(n, 1), dtype=torch.int64, device=device)[:n]
    vals = torch.empty(max(n, 1), dtype=torch.int64, device=device)[:n]
    st = stream if stream is not None else torch.cuda.current_stream(keys.device)
    rc = _L().syn_gpu_kv(family, s, n, domain, seed & (2**64 - 1), keys.data_ptr(),
                         vals.data_ptr(), st.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"syn_gpu_kv failed (cudaError {rc})")
    return keys, vals


def _unit(seed: int, j: int) -> float:
    return (_host_lib().syn_draw(seed & (2**64 - 1), TAG_INST, j) >> 11) * 2.0**-53


def instance(seed: int, rows_lo: int = 1_000_000, rows_hi: int = 50_000_000,
             dom_lo: int = 10, dom_hi: int = 100_000_000) -> dict:
    """The recipe of instance `seed`: rows, family, s, domain."""
    lr = math.log(rows_lo) + _unit(seed, 0) * (math.log(rows_hi) - math.log(rows_lo))
    ld = math.log(dom_lo) + _unit(seed, 2) * (math.log(dom_hi) - math.log(dom_lo))
    name, fam, s = FAMILIES[int(_unit(seed, 1) * len(FAMILIES))]
    return {"seed": seed, "rows": int(round(math.exp(lr))), "family": name, "fam": fam, "s": s,
            "domain": max(1, int(round(math.exp(ld))))}


def instance_kv(inst: dict, device="cuda", stream=None):
    return kv(inst["fam"], inst["s"], inst["rows"], inst["domain"], inst["seed"], device, stream)


def join_sides(n_build: int, n_probe: int, seed: int, device="cuda", stream=None,
               hit_threshold: int | None = None):
    """(build keys, build payload, probe keys) CUDA int64 tensors, the host
    generator's join streams (90 % of probe rows hit by default)."""
    import torch

    from . import HIT_90

    thr = HIT_90 if hit_threshold is None else hit_threshold
    bk = torch.empty(max(n_build, 1), dtype=torch.int64, device=device)[:n_build]
    bp = torch.empty(max(n_build, 1), dtype=torch.int64, device=device)[:n_build]
    pk = torch.empty(max(n_probe, 1), dtype=torch.int64, device=device)[:n_probe]
    st = (stream if stream is not None else torch.cuda.current_stream(bk.device)).cuda_stream
    L = _L()
    rc = L.syn_gpu_join_build(n_build, seed & (2**64 - 1), bk.data_ptr(), bp.data_ptr(), st)
    if rc == 0:
        rc = L.syn_gpu_join_probe(n_probe, max(1, n_build), thr, seed & (2**64 - 1),
                                  pk.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"join generator failed (cudaError {rc})")
    return bk, bp, pk


def batch_recipe(seed: int, n_groupby: int = 4096, n_join: int = 512) -> dict:
    """The batched workload: group-by instances with rows log-uniform in
    [1e3, 4e6], groups log-uniform in [1, 1e5], int32 keys at even and int64
    keys at odd positions; join partitions with build sides log-uniform in
    [1e3, 2.56e5] (unique keys) and probe sides log-uniform in [8e3, 2e6]
    (90 % hits)."""
    def lu(j, lo, hi):
        return int(round(math.exp(math.log(lo) + _unit(seed, j) * (math.log(hi) - math.log(lo)))))

    gb = []
    for i in range(n_groupby):
        gb.append({"rows": lu(1000 + 2 * i, 1e3, 4e6), "groups": lu(1001 + 2 * i, 1, 1e5),
                   "key_type": "int32" if i % 2 == 0 else "int64", "seed": (seed << 20) + i})
    jn = []
    for i in range(n_join):
        jn.append({"build": lu(500_000 + 2 * i, 1e3, 2.56e5),
                   "probe": lu(500_001 + 2 * i, 8e3, 2e6), "seed": (seed << 20) + 100_000 + i})
    return {"groupby": gb, "join": jn}


def batch_inputs(recipe: dict, device="cuda"):
    """Device columns of a batch recipe: ([(keys, vals)], [(bk, bp, pk)])."""
    import torch

    gb = []
    for r in recipe["groupby"]:
        k, v = kv(0, 0.0, r["rows"], r["groups"], r["seed"], device)
        if r["key_type"] == "int32":
            k = k.to(torch.int32)  # keys truncated to 32 bits
        gb.append((k, v))
    jn = [join_sides(r["build"], r["probe"], r["seed"], device) for r in recipe["join"]]
    return gb, jn
