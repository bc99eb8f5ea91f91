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
