"""Python face of the FP64 CPU oracle (``oracle/tvc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never imports it.

The C file is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/liboracle.so``.  Every function takes and returns numpy
arrays; vectors are FP64.

Parity is pinned for every function here (see tests/test_oracle_pins.py):
closed forms, brute-force unfolding, library routines (numpy einsum, SVD,
torch dtype conversions), Eq. 3's touched-memory model, Algorithm 1's
contraction count and the paper's Table 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "F64", "F32", "BF16", "E4M3", "F16", "build", "set_threads", "tvc", "tvc_exact", "tvc_grad_x", "tvc_grad_A",
    "hopm", "hopm3", "hopm_jacobi", "quantise", "decode_bf16", "decode_e4m3", "decode_f16",
    "bf16_from_f32", "e4m3_from_f32", "f16_from_f32", "dequantise", "OracleError", "dhopm_touched",
]

F64, F32, BF16, E4M3, F16 = 0, 1, 2, 3, 4
# binary16 codes travel as numpy float16 (the same bits); BF16 codes as uint16
_DTYPE_OF = {np.dtype(np.float64): F64, np.dtype(np.float32): F32,
             np.dtype(np.uint16): BF16, np.dtype(np.uint8): E4M3, np.dtype(np.float16): F16}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    """Non-zero status from an oracle routine (1 = bad argument,
    5 = zero norm, 6 = non-finite value)."""

    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics: no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
            lib.oracle_tvc.argtypes = [I, P, P, I, P, I, P, P, D, D]
            lib.oracle_tvc_exact.argtypes = [I, P, P, I, P, I, P, P]
            lib.oracle_set_threads.argtypes = [I]
            lib.oracle_set_threads.restype = I
            lib.oracle_tmc.argtypes = [I, P, P, I, P, I, P, L, P, D, D]
            lib.oracle_khatri_rao.argtypes = [P, I, P, L, P]
            lib.oracle_mttkrp.argtypes = [I, P, P, I, P, I, P, L, P]
            lib.oracle_tvc_grad_x.argtypes = [I, P, P, I, P, I, P, P]
            lib.oracle_tvc_grad_A.argtypes = [I, P, I, P, P, P]
            for f in (lib.oracle_hopm, lib.oracle_hopm3):
                f.argtypes = [I, P, P, I, P, P, I, D, P, P, P, P, P]
            lib.oracle_hopm_jacobi.argtypes = [I, P, P, I, P, P, I, D, P, P, P]
            lib.oracle_quantise.argtypes = [I, P, I, P, P, P, I]
            lib.oracle_decode_bf16.argtypes = [ctypes.c_uint16]
            lib.oracle_decode_bf16.restype = D
            lib.oracle_decode_e4m3.argtypes = [ctypes.c_uint8]
            lib.oracle_decode_e4m3.restype = D
            lib.oracle_bf16_from_f32.argtypes = [ctypes.c_float, I]
            lib.oracle_bf16_from_f32.restype = ctypes.c_uint16
            lib.oracle_e4m3_from_f32.argtypes = [ctypes.c_float]
            lib.oracle_e4m3_from_f32.restype = ctypes.c_uint8
            lib.oracle_decode_f16.argtypes = [ctypes.c_uint16]
            lib.oracle_decode_f16.restype = D
            lib.oracle_f16_from_f32.argtypes = [ctypes.c_float]
            lib.oracle_f16_from_f32.restype = ctypes.c_uint16
            lib.oracle_dhopm_touched.argtypes = [I, L, I, I, I, I]
            lib.oracle_dhopm_touched.restype = L
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops run from this thread from now on
    (results do not depend on it); returns the previous count."""
    return int(_load().oracle_set_threads(int(n)))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _tensor(A, dims):
    A = np.ascontiguousarray(A)
    if A.dtype not in _DTYPE_OF:
        raise TypeError(f"unsupported tensor dtype {A.dtype}")
    dims = A.shape if dims is None else dims
    d = _dims(dims)
    if int(np.prod(d)) != A.size:
        raise ValueError("dims do not match the tensor size")
    return A, d, _DTYPE_OF[A.dtype]


def _scales(dt, scales, n0):
    if dt == F16 and scales is None:
        return None  # binary16 without scales: value = decode(code)
    if dt in (BF16, E4M3, F16):
        if scales is None:
            raise ValueError("narrow storage needs per-slab scales")
        s = np.ascontiguousarray(np.asarray(scales, dtype=np.float32))
        if s.size != n0:
            raise ValueError("one scale per slab A[i0] is required")
        return s
    return None


def tvc(A, mode: int, x, *, dims=None, scales=None, y=None, alpha=1.0, beta=0.0) -> np.ndarray:
    """Y = alpha * (A x_mode x) + beta * Y in FP64 (shape: dims without mode)."""
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if not 0 <= mode < d.size or x.size != d[mode]:
        raise ValueError("bad mode or vector length")
    out_shape = tuple(int(n) for i, n in enumerate(d) if i != mode)
    out = (np.zeros(out_shape) if y is None else
           np.ascontiguousarray(np.asarray(y, dtype=np.float64)).reshape(out_shape).copy())
    st = _load().oracle_tvc(dt, _p(A), _p(s), int(d.size), _p(d), int(mode), _p(x), _p(out),
                            float(alpha), float(beta))
    if st:
        raise OracleError(st, "tvc")
    return out


def tvc_exact(A, mode: int, x, *, dims=None, scales=None) -> np.ndarray:
    """Y = A x_mode x with error-free transformations (compensated dot
    product Dot2, see the C source): the exact sum rounded about once, for
    measuring the error of other arithmetic."""
    A, d, dt = _tensor(A, dims)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if not 0 <= mode < d.size or x.size != int(d[mode]):
        raise ValueError("bad mode or x length")
    s = _scales(dt, scales, int(d[0]))
    y = np.zeros(int(np.prod(d)) // int(d[mode]))
    st = _load().oracle_tvc_exact(dt, _p(A), _p(s), int(d.size), _p(d), int(mode), _p(x), _p(y))
    if st:
        raise OracleError(st, "tvc_exact")
    return y.reshape(tuple(int(n) for i, n in enumerate(d) if i != mode))


def tmc(A, mode: int, X, *, dims=None, scales=None, Y=None, alpha=1.0, beta=0.0) -> np.ndarray:
    """Y = alpha * (A x_mode X) + beta * Y in FP64 for an R x n_mode matrix X
    (shape: dims with n_mode replaced by R)."""
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim != 2 or not 0 <= mode < d.size or X.shape[1] != d[mode] or X.shape[0] < 1:
        raise ValueError("bad mode or matrix shape")
    R = int(X.shape[0])
    out_shape = tuple(R if i == mode else int(n) for i, n in enumerate(d))
    out = (np.zeros(out_shape) if Y is None else
           np.ascontiguousarray(np.asarray(Y, dtype=np.float64)).reshape(out_shape).copy())
    st = _load().oracle_tmc(dt, _p(A), _p(s), int(d.size), _p(d), int(mode), _p(X), R, _p(out),
                            float(alpha), float(beta))
    if st:
        raise OracleError(st, "tmc")
    return out


def khatri_rao(mats) -> np.ndarray:
    """Columnwise Kronecker product of matrices U_m (rows_m x R): row
    (i_0, ..., i_{c-1}) (i_0 most significant) holds prod_m U_m[i_m, :]."""
    mats = [np.ascontiguousarray(np.asarray(U, dtype=np.float64)) for U in mats]
    if not mats:
        raise ValueError("need at least one matrix (R is their column count)")
    R = mats[0].shape[1]
    if any(U.ndim != 2 or U.shape[1] != R for U in mats) or R < 1:
        raise ValueError("matrices must be 2-D with the same column count")
    rows = np.array([U.shape[0] for U in mats], dtype=np.int64)
    ptrs = (ctypes.c_void_p * len(mats))(*[U.ctypes.data for U in mats])
    out = np.empty((int(np.prod(rows)), R))
    st = _load().oracle_khatri_rao(ptrs, len(mats), _p(rows), R, _p(out))
    if st:
        raise OracleError(st, "khatri_rao")
    return out


def mttkrp(A, mode: int, factors, *, R=None, dims=None, scales=None) -> np.ndarray:
    """M[i_mode, r] = sum of A times prod_{m != mode} factors[m][i_m, r]
    (factors[m]: n_m x R; factors[mode] is ignored and may be None; R is
    needed only when no other factor gives it, as for an order-1 tensor)."""
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    if not 0 <= mode < d.size or len(factors) != d.size:
        raise ValueError("bad mode or factor count")
    mats = []
    for m in range(d.size):
        if m == mode:
            mats.append(None)
            continue
        U = np.ascontiguousarray(np.asarray(factors[m], dtype=np.float64))
        if U.ndim != 2 or U.shape[0] != d[m] or (R is not None and U.shape[1] != R):
            raise ValueError("factor m must be n_m x R")
        R = U.shape[1]
        mats.append(U)
    if R is None:
        raise ValueError("R is needed when no factor other than factors[mode] is given")
    R = int(R)
    ptrs = (ctypes.c_void_p * d.size)(*[0 if U is None else U.ctypes.data for U in mats])
    M = np.empty((int(d[mode]), R))
    st = _load().oracle_mttkrp(dt, _p(A), _p(s), int(d.size), _p(d), int(mode), ptrs, R, _p(M))
    if st:
        raise OracleError(st, "mttkrp")
    return M


def tvc_grad_x(A, mode: int, gy, *, dims=None, scales=None) -> np.ndarray:
    """gx[j] = sum_{i,l} A[i][j][l] gy[i][l] (adjoint of the contraction in x)."""
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    gy = np.ascontiguousarray(np.asarray(gy, dtype=np.float64)).ravel()
    gx = np.zeros(int(d[mode]))
    st = _load().oracle_tvc_grad_x(dt, _p(A), _p(s), int(d.size), _p(d), int(mode), _p(gy), _p(gx))
    if st:
        raise OracleError(st, "tvc_grad_x")
    return gx


def tvc_grad_A(dims, mode: int, x, gy) -> np.ndarray:
    """gA[i][j][l] = gy[i][l] x[j] (adjoint of the contraction in A)."""
    d = _dims(dims)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    gy = np.ascontiguousarray(np.asarray(gy, dtype=np.float64)).ravel()
    gA = np.zeros(tuple(int(n) for n in d))
    st = _load().oracle_tvc_grad_A(int(d.size), _p(d), int(mode), _p(x), _p(gy), _p(gA))
    if st:
        raise OracleError(st, "tvc_grad_A")
    return gA


def _hopm(fn, A, xs, iters, tol, dims, scales):
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    if len(xs) != d.size:
        raise ValueError("one start vector per mode")
    x = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in xs]))
    if x.size != int(d.sum()):
        raise ValueError("start vector lengths do not match dims")
    lam = np.zeros(1)
    sweeps = np.zeros(1, dtype=np.int32)
    hist = np.zeros(max(iters, 1))
    touched = np.zeros(max(iters, 1), dtype=np.int64)
    tvcs = np.zeros(1, dtype=np.int64)
    st = fn(dt, _p(A), _p(s), int(d.size), _p(d), _p(x), int(iters), float(tol), _p(lam),
            _p(sweeps), _p(hist), _p(touched), _p(tvcs))
    offs = np.concatenate([[0], np.cumsum(d)])
    out_x = [x[offs[m]:offs[m + 1]].copy() for m in range(d.size)]
    n = int(sweeps[0])
    return dict(status=int(st), x=out_x, lam=float(lam[0]), sweeps=n, lam_hist=hist[:n].copy(),
                touched=touched[:n].copy(), tvcs=int(tvcs[0]))


def hopm(A, xs, iters: int, tol: float = 0.0, *, dims=None, scales=None) -> dict:
    """Canonical Gauss-Seidel HOPM (Section 3).  Returns a dict with x (list),
    lam, sweeps, lam_hist, touched (Eq. 3 element counts per sweep), tvcs and
    status (0, or 5 zero norm / 6 non-finite: x keeps its last valid state)."""
    return _hopm(_load().oracle_hopm, A, xs, iters, tol, dims, scales)


def hopm3(A, xs, iters: int, tol: float = 0.0, *, dims=None, scales=None) -> dict:
    """Three-buffer HOPM of Algorithm 1 (p = 1); same outputs as :func:`hopm`."""
    return _hopm(_load().oracle_hopm3, A, xs, iters, tol, dims, scales)


def hopm_jacobi(A, xs, iters: int, tol: float = 0.0, *, dims=None, scales=None) -> dict:
    """Jacobi HOPM: every z_j of a sweep from the previous sweep's vectors
    (status, x, lam, sweeps, lam_hist as for :func:`hopm`)."""
    A, d, dt = _tensor(A, dims)
    s = _scales(dt, scales, int(d[0]))
    if len(xs) != d.size:
        raise ValueError("one start vector per mode")
    x = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in xs]))
    if x.size != int(d.sum()):
        raise ValueError("start vector lengths do not match dims")
    lam = np.zeros(1)
    sweeps = np.zeros(1, dtype=np.int32)
    hist = np.zeros(max(iters, 1))
    st = _load().oracle_hopm_jacobi(dt, _p(A), _p(s), int(d.size), _p(d), _p(x), int(iters), float(tol),
                                    _p(lam), _p(sweeps), _p(hist))
    offs = np.concatenate([[0], np.cumsum(d)])
    n = int(sweeps[0])
    return dict(status=int(st), x=[x[offs[m]:offs[m + 1]].copy() for m in range(d.size)], lam=float(lam[0]),
                sweeps=n, lam_hist=hist[:n].copy())


def quantise(src, fmt: int, *, truncate: bool = False, allow_nonfinite: bool = False):
    """Per-slab quantisation of an FP32 tensor: returns (codes, scales).
    F16 codes come back as numpy float16 (the binary16 bits); with
    allow_nonfinite an F16 overflow returns the codes instead of raising."""
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float32))
    d = _dims(src.shape)
    cdt = {E4M3: np.uint8, BF16: np.uint16, F16: np.float16}.get(fmt, np.uint16)
    codes = np.zeros(src.shape, dtype=cdt)
    scales = np.zeros(int(d[0]), dtype=np.float32)
    st = _load().oracle_quantise(int(fmt), _p(src), int(d.size), _p(d), _p(codes), _p(scales),
                                 int(bool(truncate)))
    if st and not (allow_nonfinite and fmt == F16 and st == 6):
        raise OracleError(st, "quantise")
    return codes, scales


def decode_bf16(code: int) -> float:
    return _load().oracle_decode_bf16(int(code))


def decode_e4m3(code: int) -> float:
    return _load().oracle_decode_e4m3(int(code))


def bf16_from_f32(f: float, truncate: bool = False) -> int:
    return int(_load().oracle_bf16_from_f32(float(f), int(bool(truncate))))


def e4m3_from_f32(f: float) -> int:
    return int(_load().oracle_e4m3_from_f32(float(f)))


def decode_f16(code: int) -> float:
    return _load().oracle_decode_f16(int(code))


def f16_from_f32(f: float) -> int:
    return int(_load().oracle_f16_from_f32(float(f)))


def dequantise(codes, scales) -> np.ndarray:
    """FP64 values scale[i0] * decode(code) of a narrow tensor (via the
    oracle's own decoders, one code at a time through a 256/65536 table)."""
    codes = np.asarray(codes)
    if codes.dtype == np.uint8:
        table = np.array([decode_e4m3(c) for c in range(256)])
    elif codes.dtype == np.uint16:
        table = np.array([decode_bf16(c) for c in range(65536)])
    elif codes.dtype == np.float16:
        table = np.array([decode_f16(c) for c in range(65536)])
        codes = codes.view(np.uint16)
    else:
        raise TypeError("codes must be uint8 (E4M3), uint16 (BF16) or float16 (F16)")
    vals = table[codes]
    s = np.asarray(scales, dtype=np.float64).reshape((-1,) + (1,) * (codes.ndim - 1))
    return vals * s


def dhopm_touched(d: int, n: int, p: int, s: int, j: int, three: bool = False) -> int:
    """Touched elements of one process in external iteration j of the
    distributed HOPM on n^d split along s over p processes (n % p == 0):
    the canonical chain, or Algorithm 1's with three=True."""
    r = int(_load().oracle_dhopm_touched(int(d), int(n), int(p), int(s), int(j), int(bool(three))))
    if r < 0:
        raise ValueError("invalid distributed-HOPM shape")
    return r
