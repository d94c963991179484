"""Device-side fill of the synthetic inputs (library synth/_lib/libtvc_synth.so).

Produces on the GPU exactly the bits that :mod:`synth` produces on the host
for the same (seed, stream, element index), so that tensors too large to make
on the host can be filled in place while the oracle still draws its inputs
from the host generator.  Holds none of the contraction's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth_fill.cu")
LIB = os.path.join(_HERE, "_lib", "libtvc_synth.so")
_lock = threading.Lock()
_lib = None

KINDS = {"u64": 0, "u32": 1, "gauss": 2, "lognormal": 3, "planted": 4}


def build() -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(_SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a",
                               "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} missing: run synth.device.build()")
            lib = ctypes.CDLL(LIB)
            P = ctypes.c_void_p
            lib.synth_fill.argtypes = [P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.synth_fill.restype = ctypes.c_int
            _lib = lib
    return _lib


def fill(out: torch.Tensor, kind: str, seed: int, sid: int = 0, offset: int = 0, dims=None, us=None,
         stream=None) -> torch.Tensor:
    """Fill the contiguous float32/float64 CUDA tensor ``out`` with elements
    offset .. offset+numel-1 of the given stream (see :func:`synth.tensor`)."""
    if out.dtype not in (torch.float32, torch.float64) or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32/float64 CUDA tensor")
    lib = _load()
    k = KINDS[kind]
    dims_arr = None
    us_arr = None
    keep = []
    if k == KINDS["planted"]:
        dims = [int(n) for n in dims]
        dims_arr = (ctypes.c_int64 * len(dims))(*dims)
        ut = [torch.as_tensor(u, dtype=torch.float64).to(out.device).contiguous() for u in us]
        keep = ut
        us_arr = (ctypes.c_void_p * len(ut))(*[u.data_ptr() for u in ut])
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rc = lib.synth_fill(ctypes.c_void_p(out.data_ptr()), int(out.dtype == torch.float32), out.numel(), int(offset),
                        int(seed), int(sid), k, len(dims) if dims else 0, dims_arr, us_arr, ctypes.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"synth_fill failed: cudaError {rc}")
    if keep:
        torch.cuda.current_stream().synchronize()
    return out
