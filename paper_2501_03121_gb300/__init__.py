"""GB300-native tensor-vector contraction (TVC) and higher-order power method.

Thin Python binding over the C ABI of ``include/tvc.h`` (library
``_lib/libtvc_gb300.so``, built by ``build.py``).  Every step of the
computation runs in the CUDA kernels of that library; this module only
marshals torch tensors (device memory, streams) into pointers and sizes.
There is no CPU fallback: if the library is missing, every call raises.

Method: Martinez-Ferrer, Yzelman, Beltran, "Distributed and heterogeneous
tensor-vector contraction algorithms for high performance computing"
(arXiv 2501.03121).
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

__all__ = [
    "F64", "F32", "BF16", "E4M3", "F16", "F32D", "TVCError", "load_library", "tvc", "tvc_workspace_size",
    "dtype_code", "library_path", "kernel_launches", "hopm", "hopm_workspace_size", "HopmResult", "quantise", "tvc_backward", "TVCFunction", "tvc_autograd", "hopm_backward", "HOPMFunction", "hopm_autograd", "TVCBatch", "HOPMBatch", "BATCH_PREUPLOADED",
    "split_1d", "slab_extract", "slab_insert", "split_tensor", "dtvc", "dtvc_workspace_size", "dhopm",
    "dhopm_workspace_size", "hopm_jacobi",
]

F64, F32, BF16, E4M3, F16, F32D = 0, 1, 2, 3, 4, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_lib", "libtvc_gb300.so")
_lock = threading.Lock()
_lib = None


class TVCError(RuntimeError):
    """Non-zero tvc_status from the library."""

    def __init__(self, status: int, where: str):
        msg = _status_string(status)
        super().__init__(f"{where}: {msg}")
        self.status = status


def _status_string(status: int) -> str:
    try:
        return load_library().tvc_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - library unavailable
        return f"status {status}"


def load_library():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(library_path):
            raise RuntimeError(
                f"CUDA library {library_path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(library_path)
        P, I, D, Z, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_int64
        lib.tvc_status_string.argtypes = [I]
        lib.tvc_status_string.restype = ctypes.c_char_p
        lib.tvc.argtypes = [P, I, P, I, P, P, I, P]
        lib.tvc.restype = I
        lib.tvc_ex.argtypes = [P, I, P, I, P, P, I, P, D, D, P, Z, P]
        lib.tvc_ex.restype = I
        lib.tvc_workspace_size.argtypes = [I, P, I, I]
        lib.tvc_workspace_size.restype = Z
        lib.tmc.argtypes = [P, I, P, I, P, L, P, I, P, D, D, P, Z, P]
        lib.tmc.restype = I
        lib.tmc_workspace_size.argtypes = [I, P, I, L, I]
        lib.tmc_workspace_size.restype = Z
        lib.khatri_rao.argtypes = [P, I, P, L, P, I, P]
        lib.khatri_rao.restype = I
        lib.mttkrp.argtypes = [P, I, P, I, P, L, P, I, P, P, Z, P]
        lib.mttkrp.restype = I
        lib.mttkrp_workspace_size.argtypes = [I, P, I, L, I]
        lib.mttkrp_workspace_size.restype = Z
        lib.hopm.argtypes = [P, I, P, P, I, D, P, P, P, P, I, P, P, Z, P]
        lib.hopm.restype = I
        lib.hopm_workspace_size.argtypes = [I, P, I]
        lib.hopm_workspace_size.restype = Z
        lib.hopm_jacobi.argtypes = [P, I, P, P, I, D, P, P, P, P, I, P, P, Z, P]
        lib.hopm_jacobi.restype = I
        lib.hopm_jacobi_workspace_size.argtypes = [I, P, I]
        lib.hopm_jacobi_workspace_size.restype = Z
        lib.tvc_quantise.argtypes = [P, I, P, I, P, P, I, P, P, Z, P]
        lib.tvc_quantise.restype = I
        lib.tvc_quantise_workspace_size.argtypes = [I, P]
        lib.tvc_quantise_workspace_size.restype = Z
        lib.tvc_backward.argtypes = [P, I, P, I, P, P, P, P, I, P, D, P, Z, P]
        lib.tvc_backward.restype = I
        lib.tvc_backward_workspace_size.argtypes = [I, P, I, I]
        lib.tvc_backward_workspace_size.restype = Z
        lib.hopm_backward.argtypes = [P, I, P, P, I, P, P, P, P, I, P, P, Z, P]
        lib.hopm_backward.restype = I
        lib.hopm_backward_workspace_size.argtypes = [I, P, I, I]
        lib.hopm_backward_workspace_size.restype = Z
        lib.tvc_batched.argtypes = [P, I, I, P, Z, P]
        lib.tvc_batched.restype = I
        lib.tvc_batched_workspace_size.argtypes = [P, I]
        lib.tvc_batched_workspace_size.restype = Z
        lib.tvc_batched_autotune.argtypes = [P, I, P, Z, P]
        lib.tvc_batched_autotune.restype = I
        lib.hopm_batched.argtypes = [P, I, I, I, P, Z, P]
        lib.hopm_batched.restype = I
        lib.hopm_batched_workspace_size.argtypes = [P, I]
        lib.hopm_batched_workspace_size.restype = Z
        lib.tvc_split_1d.argtypes = [L, I, L, P]
        lib.tvc_split_1d.restype = I
        lib.tvc_slab_copy.argtypes = [P, P, I, P, I, L, L, Z, I, P]
        lib.tvc_slab_copy.restype = I
        lib.dtvc.argtypes = [P, I, P, I, P, I, I, P, P, I, P, D, D, P, Z, P]
        lib.dtvc.restype = I
        lib.dtvc_workspace_size.argtypes = [I, P, I, P, I, I, I]
        lib.dtvc_workspace_size.restype = Z
        lib.dhopm.argtypes = [P, I, P, I, P, I, P, I, D, P, P, P, P, I, P, P, Z, P]
        lib.dhopm.restype = I
        lib.dhopm_workspace_size.argtypes = [I, P, I, P, I, I]
        lib.dhopm_workspace_size.restype = Z
        lib.tvc_read_status.argtypes = [P, P, P]
        lib.tvc_read_status.restype = I
        lib.tvc_kernel_launches.argtypes = []
        lib.tvc_kernel_launches.restype = ctypes.c_uint64
        _lib = lib
        return lib


_TORCH_CODE = {
    torch.float64: F64,
    torch.float32: F32,
    torch.bfloat16: BF16,
    torch.uint16: BF16,
    torch.float8_e4m3fn: E4M3,
    torch.uint8: E4M3,
    torch.float16: F16,
}


def dtype_code(t: torch.Tensor) -> int:
    """Storage code of a tensor: float64, float32, bfloat16 (or raw uint16
    codes), float8_e4m3fn (or raw uint8 codes), float16 (binary16 codes)."""
    try:
        return _TORCH_CODE[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported tensor dtype {t.dtype}") from None


def vec_dtype(code: int) -> torch.dtype:
    return torch.float64 if code in (F64, F32D) else torch.float32


def _with_vectors(code: int, vec: torch.Tensor | None) -> int:
    """FP32 storage with float64 vectors selects single-double (F32D: FP64
    arithmetic on binary32 elements, Section 5.5)."""
    if code == F32 and vec is not None and vec.dtype == torch.float64:
        return F32D
    return code


def _dims_array(shape):
    arr = (ctypes.c_int64 * max(1, len(shape)))(*[int(n) for n in shape])
    return arr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(status, where):
    if status != 0:
        raise TVCError(status, where)


def _check_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("tensors must be contiguous CUDA tensors")


def read_status(status: torch.Tensor, *, stream=None) -> int:
    """Value of a device status word (one int32 on the GPU) once the work
    queued before it on `stream` has finished: a tvc_status code."""
    lib = load_library()
    if status.dtype != torch.int32 or status.numel() < 1:
        raise ValueError("status must be a CUDA int32 tensor")
    _check_cuda(status)
    out = ctypes.c_int(0)
    _check(lib.tvc_read_status(_ptr(status), ctypes.byref(out), _stream(stream)), "tvc_read_status")
    return int(out.value)


def kernel_launches() -> int:
    """Kernels the library has launched so far in this process."""
    return int(load_library().tvc_kernel_launches())


def tvc_workspace_size(shape, mode: int, code: int) -> int:
    """Bytes of workspace tvc(..., workspace=...) needs for this shape."""
    lib = load_library()
    dims = _dims_array(shape)
    return int(lib.tvc_workspace_size(len(shape), dims, int(mode), int(code)))


def tvc(A: torch.Tensor, mode: int, x: torch.Tensor, *, y: torch.Tensor | None = None,
        scales: torch.Tensor | None = None, alpha: float = 1.0, beta: float = 0.0,
        workspace: torch.Tensor | None = None, stream=None, shape=None) -> torch.Tensor:
    """Y = alpha * (A x_mode x) + beta * Y on the GPU.

    ``A`` holds the tensor (its shape, or ``shape`` for raw uint8/uint16
    codes given flat); ``x`` is float64 for float64 storage and float32
    otherwise.  ``scales`` are the n_0 per-slab FP32 scales of narrow
    storage.  Without ``workspace`` (and with alpha=1, beta=0, no scales)
    the library's own workspace is used.
    """
    lib = load_library()
    code = _with_vectors(dtype_code(A), x)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    if not 0 <= mode < len(shape):
        raise ValueError("mode out of range")
    vt = vec_dtype(code)
    if x.dtype != vt or x.numel() != shape[mode]:
        raise ValueError(f"x must be {vt} with {shape[mode]} entries")
    out_shape = tuple(n for i, n in enumerate(shape) if i != mode)
    if y is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs y")
        y = torch.empty(out_shape, dtype=vt, device=A.device)
    elif y.dtype != vt or y.numel() != math.prod(out_shape):
        raise ValueError("y has the wrong dtype or size")
    if scales is not None and scales.dtype != torch.float32:
        raise ValueError("scales must be float32")
    _check_cuda(A, x, y, scales, workspace)
    dims = _dims_array(shape)
    st = _stream(stream)
    if workspace is None and scales is None and alpha == 1.0 and beta == 0.0:
        status = lib.tvc(_ptr(A), len(shape), dims, int(mode), _ptr(x), _ptr(y), code, st)
    else:
        if workspace is None:
            need = lib.tvc_workspace_size(len(shape), dims, int(mode), code)
            workspace = torch.empty(max(1, need), dtype=torch.uint8, device=A.device)
        status = lib.tvc_ex(_ptr(A), len(shape), dims, int(mode), _ptr(x), _ptr(y), code, _ptr(scales),
                            float(alpha), float(beta), _ptr(workspace), workspace.numel(), st)
    _check(status, "tvc")
    return y


def tmc_workspace_size(shape, mode: int, R: int, code: int) -> int:
    """Bytes of workspace tmc(..., workspace=...) needs for this shape and R."""
    lib = load_library()
    return int(lib.tmc_workspace_size(len(shape), _dims_array(shape), int(mode), int(R), int(code)))


def tmc(A: torch.Tensor, mode: int, X: torch.Tensor, *, Y: torch.Tensor | None = None,
        scales: torch.Tensor | None = None, alpha: float = 1.0, beta: float = 0.0,
        workspace: torch.Tensor | None = None, stream=None, shape=None) -> torch.Tensor:
    """Y = alpha * (A x_mode X) + beta * Y on the GPU for an R x n_mode matrix X
    (float64 for float64 storage, float32 otherwise; float64 with float32
    storage selects single-double).  Y has the shape of A with n_mode
    replaced by R."""
    lib = load_library()
    code = _with_vectors(dtype_code(A), X)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    if not 0 <= mode < len(shape):
        raise ValueError("mode out of range")
    vt = vec_dtype(code)
    if X.dtype != vt or X.dim() != 2 or X.shape[1] != shape[mode] or X.shape[0] < 1 or not X.is_contiguous():
        raise ValueError(f"X must be a contiguous {vt} matrix with {shape[mode]} columns")
    R = int(X.shape[0])
    out_shape = tuple(R if i == mode else n for i, n in enumerate(shape))
    if Y is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs Y")
        Y = torch.empty(out_shape, dtype=vt, device=A.device)
    elif Y.dtype != vt or Y.numel() != math.prod(out_shape) or not Y.is_contiguous():
        raise ValueError("Y has the wrong dtype or size")
    if scales is not None and scales.dtype != torch.float32:
        raise ValueError("scales must be float32")
    _check_cuda(A, X, Y, scales, workspace)
    dims = _dims_array(shape)
    if workspace is None:
        need = lib.tmc_workspace_size(len(shape), dims, int(mode), R, code)
        if need:
            workspace = torch.empty(need, dtype=torch.uint8, device=A.device)
    status = lib.tmc(_ptr(A), len(shape), dims, int(mode), _ptr(X), R, _ptr(Y), code, _ptr(scales), float(alpha),
                     float(beta), _ptr(workspace), 0 if workspace is None else workspace.numel(), _stream(stream))
    _check(status, "tmc")
    return Y


def khatri_rao(mats, *, stream=None) -> torch.Tensor:
    """Columnwise Kronecker product U_0 (.) U_1 (.) ... of CUDA matrices
    (rows_m x R, all float64 or all float32): row (i_0, ..., i_{c-1}), i_0
    most significant, holds prod_m U_m[i_m, :]."""
    lib = load_library()
    mats = list(mats)
    if not mats:
        raise ValueError("need at least one matrix")
    dt = mats[0].dtype
    R = int(mats[0].shape[1]) if mats[0].dim() == 2 else -1
    if dt not in (torch.float64, torch.float32) or any(
            U.dtype != dt or U.dim() != 2 or U.shape[1] != R or not U.is_contiguous() for U in mats):
        raise ValueError("matrices must be contiguous 2-D float64 or float32 with one column count")
    _check_cuda(*mats)
    rows = (ctypes.c_int64 * len(mats))(*[int(U.shape[0]) for U in mats])
    ptrs = (ctypes.c_void_p * len(mats))(*[U.data_ptr() for U in mats])
    out = torch.empty((math.prod(int(U.shape[0]) for U in mats), R), dtype=dt, device=mats[0].device)
    _check(lib.khatri_rao(ptrs, len(mats), rows, R, _ptr(out), F64 if dt == torch.float64 else F32,
                          _stream(stream)), "khatri_rao")
    return out


def mttkrp_workspace_size(shape, mode: int, R: int, code: int) -> int:
    """Bytes of workspace mttkrp(..., workspace=...) needs."""
    lib = load_library()
    return int(lib.mttkrp_workspace_size(len(shape), _dims_array(shape), int(mode), int(R), int(code)))


def mttkrp(A: torch.Tensor, mode: int, factors, *, R: int | None = None, scales: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None, stream=None, shape=None) -> torch.Tensor:
    """Matricized tensor times Khatri-Rao product on the GPU:
    M[i_mode, r] = sum of A times prod_{m != mode} factors[m][i_m, r].
    factors: one n_m x R CUDA matrix per mode (factors[mode] ignored, may be
    None); float64 for float64 storage, float32 otherwise (float64 with
    float32 storage selects single-double).  Returns M (n_mode x R)."""
    lib = load_library()
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    d = len(shape)
    if not 0 <= mode < d or len(factors) != d:
        raise ValueError("bad mode or factor count")
    others = [factors[m] for m in range(d) if m != mode]
    vref = others[0] if others else None
    code = _with_vectors(dtype_code(A), vref)
    vt = vec_dtype(code)
    if others:
        R = int(others[0].shape[1])
    elif R is None:
        raise ValueError("R is needed when no factor other than factors[mode] is given")
    for m in range(d):
        if m == mode:
            continue
        U = factors[m]
        if U.dtype != vt or U.dim() != 2 or tuple(U.shape) != (shape[m], R) or not U.is_contiguous():
            raise ValueError(f"factor {m} must be a contiguous {vt} matrix of shape ({shape[m]}, {R})")
    if scales is not None and scales.dtype != torch.float32:
        raise ValueError("scales must be float32")
    _check_cuda(A, scales, workspace, *others)
    dims = _dims_array(shape)
    if workspace is None:
        need = lib.mttkrp_workspace_size(d, dims, int(mode), R, code)
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=A.device)
    M = torch.empty((shape[mode], R), dtype=vt, device=A.device)
    ptrs = (ctypes.c_void_p * d)(*[0 if (m == mode or factors[m] is None) else factors[m].data_ptr()
                                   for m in range(d)])
    _check(lib.mttkrp(_ptr(A), d, dims, int(mode), ptrs, R, _ptr(M), code, _ptr(scales), _ptr(workspace),
                      workspace.numel(), _stream(stream)), "mttkrp")
    return M


class HopmResult:
    """Device outputs of :func:`hopm` (all torch tensors on the GPU)."""

    def __init__(self, xs, lam, sweeps, status, lam_hist):
        self.x = xs
        self.lam = lam
        self.sweeps = sweeps
        self.status = status
        self.lam_hist = lam_hist

    def check(self):
        st = int(self.status.item())
        if st != 0:
            raise TVCError(st, "hopm (device status)")
        return self


def hopm_workspace_size(shape, code: int) -> int:
    lib = load_library()
    return int(lib.hopm_workspace_size(len(shape), _dims_array(shape), int(code)))


def hopm(A: torch.Tensor, xs, iters: int, tol: float = 0.0, *, scales: torch.Tensor | None = None,
         workspace: torch.Tensor | None = None, stream=None, shape=None, inplace: bool = False) -> HopmResult:
    """Higher-order power method on the GPU (Gauss-Seidel sweeps of
    x_j = A x_{m != j} x_m / ||.||).  ``xs`` are the start vectors (x[0] is
    not read); unless ``inplace`` they are copied first.  Returns device
    tensors: x, lam, sweeps, status, lam_hist (lambda per completed sweep)."""
    lib = load_library()
    code = _with_vectors(dtype_code(A), xs[-1] if len(xs) else None)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    if len(shape) < 2 or len(xs) != len(shape):
        raise ValueError("hopm needs order >= 2 and one start vector per mode")
    vt = vec_dtype(code)
    xs = [v if inplace else v.clone() for v in xs]
    for m, v in enumerate(xs):
        if v.dtype != vt or v.numel() != shape[m]:
            raise ValueError(f"x[{m}] must be {vt} with {shape[m]} entries")
    _check_cuda(A, scales, workspace, *xs)
    dev = A.device
    lam = torch.zeros(1, dtype=torch.float64, device=dev)
    sweeps = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    hist = torch.zeros(max(1, iters), dtype=torch.float64, device=dev)
    dims = _dims_array(shape)
    if workspace is None:
        need = lib.hopm_workspace_size(len(shape), dims, code)
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    ptrs = (ctypes.c_void_p * len(xs))(*[v.data_ptr() for v in xs])
    st = lib.hopm(_ptr(A), len(shape), dims, ptrs, int(iters), float(tol), _ptr(lam), _ptr(sweeps), _ptr(status),
                  _ptr(hist), code, _ptr(scales), _ptr(workspace), workspace.numel(), _stream(stream))
    _check(st, "hopm")
    return HopmResult(xs, lam, sweeps, status, hist)


def hopm_jacobi(A: torch.Tensor, xs, iters: int, tol: float = 0.0, *, scales: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, stream=None, shape=None, inplace: bool = False) -> HopmResult:
    """Jacobi HOPM on the GPU: every update of a sweep from the previous
    sweep's vectors (see include/tvc.h); outputs as for :func:`hopm`."""
    lib = load_library()
    code = _with_vectors(dtype_code(A), xs[-1] if len(xs) else None)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    if len(shape) < 2 or len(xs) != len(shape):
        raise ValueError("hopm_jacobi needs order >= 2 and one start vector per mode")
    vt = vec_dtype(code)
    xs = [v if inplace else v.clone() for v in xs]
    for m, v in enumerate(xs):
        if v.dtype != vt or v.numel() != shape[m]:
            raise ValueError(f"x[{m}] must be {vt} with {shape[m]} entries")
    _check_cuda(A, scales, workspace, *xs)
    dev = A.device
    lam = torch.zeros(1, dtype=torch.float64, device=dev)
    sweeps = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    hist = torch.zeros(max(1, iters), dtype=torch.float64, device=dev)
    dims = _dims_array(shape)
    if workspace is None:
        need = lib.hopm_jacobi_workspace_size(len(shape), dims, code)
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    ptrs = (ctypes.c_void_p * len(xs))(*[v.data_ptr() for v in xs])
    st = lib.hopm_jacobi(_ptr(A), len(shape), dims, ptrs, int(iters), float(tol), _ptr(lam), _ptr(sweeps),
                         _ptr(status), _ptr(hist), code, _ptr(scales), _ptr(workspace), workspace.numel(),
                         _stream(stream))
    _check(st, "hopm_jacobi")
    return HopmResult(xs, lam, sweeps, status, hist)


def quantise(src: torch.Tensor, code: int, *, truncate: bool = False, stream=None):
    """Per-slab quantisation of a float32 CUDA tensor to BF16 (uint16 codes),
    E4M3 (uint8 codes) or F16 (float16 codes); returns (codes, scales,
    status) on the device."""
    lib = load_library()
    if src.dtype != torch.float32:
        raise ValueError("src must be float32")
    if code not in (BF16, E4M3, F16):
        raise ValueError("code must be BF16, E4M3 or F16")
    _check_cuda(src)
    shape = tuple(src.shape)
    dims = _dims_array(shape)
    cdt = {E4M3: torch.uint8, BF16: torch.uint16, F16: torch.float16}[code]
    codes = torch.empty(shape, dtype=cdt, device=src.device)
    scales = torch.empty(shape[0], dtype=torch.float32, device=src.device)
    status = torch.zeros(1, dtype=torch.int32, device=src.device)
    ws = torch.empty(max(1, lib.tvc_quantise_workspace_size(len(shape), dims)), dtype=torch.uint8, device=src.device)
    st = lib.tvc_quantise(_ptr(src), len(shape), dims, code, _ptr(codes), _ptr(scales), int(bool(truncate)),
                          _ptr(status), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "quantise")
    return codes, scales, status


def tvc_backward(A: torch.Tensor | None, mode: int, x: torch.Tensor | None, gy: torch.Tensor, *, need_x: bool = True,
                 need_A: bool = True, scales: torch.Tensor | None = None, gA: torch.Tensor | None = None,
                 beta_A: float = 0.0, shape=None, code: int | None = None, stream=None):
    """Adjoints of Y = A x_mode x: returns (gx, gA) (None where not asked).
    gx = sum_{i,l} A[i,j,l] gy[i,l]; gA = gy (x) x along mode (+ beta_A gA)."""
    lib = load_library()
    if code is None:
        code = _with_vectors(dtype_code(A), gy)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    vt = vec_dtype(code)
    dev = gy.device
    N = math.prod(shape)
    if gy.dtype != vt or gy.numel() != N // shape[mode]:
        raise ValueError("gy has the wrong dtype or size")
    gx = torch.empty(shape[mode], dtype=vt, device=dev) if need_x else None
    if need_A and gA is None:
        gA = torch.empty(shape, dtype=vt, device=dev)
    if not need_A:
        gA = None
    _check_cuda(A, x, gy, gx, gA, scales)
    dims = _dims_array(shape)
    need = lib.tvc_backward_workspace_size(len(shape), dims, int(mode), code) if need_x else 0
    ws = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    st = lib.tvc_backward(_ptr(A), len(shape), dims, int(mode), _ptr(x), _ptr(gy), _ptr(gx), _ptr(gA), code,
                          _ptr(scales), float(beta_A), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "tvc_backward")
    return gx, gA


class TVCFunction(torch.autograd.Function):
    """Autograd wrapper of the contraction: forward tvc(), backward
    tvc_backward() (gradient for x always; for A when A is a float tensor
    that requires grad; narrow codes carry no gradient)."""

    @staticmethod
    def forward(ctx, A, x, mode, scales=None):
        ctx.mode = int(mode)
        ctx.save_for_backward(A, x, scales)
        return tvc(A, ctx.mode, x, scales=scales)

    @staticmethod
    def backward(ctx, gy):
        A, x, scales = ctx.saved_tensors
        need_x = ctx.needs_input_grad[1]
        need_A = ctx.needs_input_grad[0] and A.is_floating_point() and A.dtype in (torch.float64, torch.float32)
        gy = gy.contiguous()
        gx, gA = tvc_backward(A, ctx.mode, x, gy, need_x=need_x, need_A=need_A, scales=scales)
        if gA is not None and gA.dtype != A.dtype:  # single-double: FP64 gradient of FP32 storage
            gA = gA.to(A.dtype)
        return gA, gx, None, None


def tvc_autograd(A, x, mode, scales=None):
    """Differentiable y = A x_mode x (see :class:`TVCFunction`)."""
    return TVCFunction.apply(A, x, mode, scales)


def hopm_backward(A: torch.Tensor, x0, iters: int, gx_final=None, g_lambda: torch.Tensor | None = None, *,
                  scales: torch.Tensor | None = None, shape=None, stream=None):
    """Gradients of `iters` HOPM sweeps from start vectors x0: returns
    (gA, gstart) given upstream gradients of the final vectors (list,
    entries may be None) and of lambda (1-element float64 device tensor)."""
    lib = load_library()
    code = _with_vectors(dtype_code(A), x0[-1] if len(x0) else None)
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    vt = vec_dtype(code)
    d = len(shape)
    dev = A.device
    x0 = [v.contiguous() for v in x0]
    gA = torch.empty(shape, dtype=vt, device=dev)
    gstart = [torch.zeros(n, dtype=vt, device=dev) for n in shape]
    gfin = [None] * d if gx_final is None else [None if g is None else g.contiguous() for g in gx_final]
    if g_lambda is not None:
        g_lambda = g_lambda.to(device=dev, dtype=torch.float64).reshape(1).contiguous()
    _check_cuda(A, scales, *x0, *[g for g in gfin if g is not None])
    dims = _dims_array(shape)
    need = lib.hopm_backward_workspace_size(d, dims, code, int(iters))
    ws = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    P = ctypes.c_void_p
    x0p = (P * d)(*[v.data_ptr() for v in x0])
    gfp = (P * d)(*[(g.data_ptr() if g is not None else None) for g in gfin])
    gsp = (P * d)(*[g.data_ptr() for g in gstart])
    st = lib.hopm_backward(_ptr(A), d, dims, x0p, int(iters), gfp, _ptr(g_lambda), _ptr(gA), gsp, code,
                           _ptr(scales), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "hopm_backward")
    return gA, gstart


class HOPMFunction(torch.autograd.Function):
    """Autograd wrapper of a fixed-count HOPM: forward returns (lambda,
    x_0, ..., x_{d-1}); backward recomputes the sweeps (see hopm_backward)."""

    @staticmethod
    def forward(ctx, A, iters, *x0):
        ctx.iters = int(iters)
        ctx.save_for_backward(A, *x0)
        r = hopm(A, list(x0), ctx.iters, 0.0).check()
        return (r.lam.clone(),) + tuple(r.x)

    @staticmethod
    def backward(ctx, g_lam, *gxs):
        A, *x0 = ctx.saved_tensors
        gA, gstart = hopm_backward(A, x0, ctx.iters, list(gxs), g_lam)
        if gA.dtype != A.dtype:  # single-double: FP64 gradient of FP32 storage
            gA = gA.to(A.dtype)
        return (gA, None) + tuple(gstart)


def hopm_autograd(A, x0, iters):
    """Differentiable (lambda, x_0..x_{d-1}) of `iters` HOPM sweeps."""
    return HOPMFunction.apply(A, iters, *x0)


MAX_ORDER = 16
BATCH_PREUPLOADED = 1


class _TvcBatchDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("order", ctypes.c_int), ("mode", ctypes.c_int),
                ("dims", ctypes.c_int64 * MAX_ORDER), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("gy", ctypes.c_void_p), ("gx", ctypes.c_void_p), ("gA", ctypes.c_void_p)]


class _HopmBatchDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("order", ctypes.c_int), ("dims", ctypes.c_int64 * MAX_ORDER),
                ("x", ctypes.c_void_p * MAX_ORDER), ("lambda_out", ctypes.c_void_p), ("status_out", ctypes.c_void_p)]


def _p(t):
    return None if t is None else t.data_ptr()


class TVCBatch:
    """A batch of FP32 contractions (+ adjoints) run by one persistent
    launch.  items: dicts with A (float32 CUDA tensor), mode, x, and any of
    y / gy, gx / gA (outputs preallocated by the caller; None to skip).
    The descriptors are uploaded once (first run); later runs reuse them
    and can be captured in a CUDA graph."""

    def __init__(self, items):
        self.items = items
        n = len(items)
        arr = (_TvcBatchDesc * max(1, n))()
        for b, it in enumerate(items):
            A = it["A"]
            shape = tuple(it.get("shape") or A.shape)
            d = arr[b]
            d.A = _p(A)
            d.order = len(shape)
            d.mode = int(it["mode"])
            for m, v in enumerate(shape):
                d.dims[m] = int(v)
            d.x, d.y, d.gy, d.gx, d.gA = (_p(it.get(k)) for k in ("x", "y", "gy", "gx", "gA"))
        self._arr = arr
        self.count = n
        lib = load_library()
        dev = items[0]["A"].device if items else torch.device("cuda")
        need = lib.tvc_batched_workspace_size(arr, n)
        self.workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
        self._uploaded = False

    def autotune(self, stream=None):
        lib = load_library()
        _check(lib.tvc_batched_autotune(self._arr, self.count, _ptr(self.workspace), self.workspace.numel(),
                                        _stream(stream)), "tvc_batched_autotune")
        self._uploaded = False  # choices changed: upload again

    def run(self, stream=None):
        lib = load_library()
        flags = BATCH_PREUPLOADED if self._uploaded else 0
        _check(lib.tvc_batched(self._arr, self.count, flags, _ptr(self.workspace), self.workspace.numel(),
                               _stream(stream)), "tvc_batched")
        self._uploaded = True


class HOPMBatch:
    """A batch of FP32 power methods (one block per tensor, `iters` sweeps)."""

    def __init__(self, items, iters):
        self.iters = int(iters)
        n = len(items)
        arr = (_HopmBatchDesc * max(1, n))()
        for b, it in enumerate(items):
            A = it["A"]
            shape = tuple(it.get("shape") or A.shape)
            d = arr[b]
            d.A = _p(A)
            d.order = len(shape)
            for m, v in enumerate(shape):
                d.dims[m] = int(v)
                d.x[m] = _p(it["x"][m])
            d.lambda_out = _p(it.get("lam"))
            d.status_out = _p(it.get("status"))
        self._arr = arr
        self.count = n
        lib = load_library()
        dev = items[0]["A"].device if items else torch.device("cuda")
        need = lib.hopm_batched_workspace_size(arr, n)
        self.workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
        self._uploaded = False

    def run(self, stream=None):
        lib = load_library()
        flags = BATCH_PREUPLOADED if self._uploaded else 0
        _check(lib.hopm_batched(self._arr, self.count, self.iters, flags, _ptr(self.workspace),
                                self.workspace.numel(), _stream(stream)), "hopm_batched")
        self._uploaded = True


# ------------------------------------------------ 1D split, virtual ranks


def split_1d(n: int, p: int, quantum: int = 1) -> list:
    """Slab boundaries [0, ..., n] of the 1D split of a dimension of n
    entries over p ranks (ceil(n/p) rounded up to a multiple of `quantum`;
    p may come out lower).  Host only."""
    lib = load_library()
    starts = (ctypes.c_int64 * (int(p) + 1))()
    r = lib.tvc_split_1d(int(n), int(p), int(quantum), starts)
    if r < 0:
        raise ValueError(f"invalid split: n={n}, p={p}, quantum={quantum}")
    return [int(starts[i]) for i in range(r + 1)]


def _slab_shape(shape, s, start, end):
    return tuple((end - start) if i == s else n for i, n in enumerate(shape))


def slab_extract(A: torch.Tensor, s: int, start: int, end: int, *, shape=None, stream=None) -> torch.Tensor:
    """Dense copy of the slab [start, end) of A along dimension s."""
    lib = load_library()
    shape = tuple(A.shape) if shape is None else tuple(int(n) for n in shape)
    out = torch.empty(_slab_shape(shape, s, start, end), dtype=A.dtype, device=A.device)
    _check_cuda(A, out)
    _check(lib.tvc_slab_copy(_ptr(A), _ptr(out), len(shape), _dims_array(shape), int(s), int(start), int(end),
                             A.element_size(), 0, _stream(stream)), "tvc_slab_copy")
    return out


def slab_insert(slab: torch.Tensor, out: torch.Tensor, s: int, start: int, end: int, *, shape=None,
                stream=None) -> torch.Tensor:
    """Writes a dense slab into the range [start, end) of `out` along s."""
    lib = load_library()
    shape = tuple(out.shape) if shape is None else tuple(int(n) for n in shape)
    if slab.dtype != out.dtype or slab.numel() != math.prod(_slab_shape(shape, s, start, end)):
        raise ValueError("slab does not match the range")
    _check_cuda(slab, out)
    _check(lib.tvc_slab_copy(_ptr(slab), _ptr(out), len(shape), _dims_array(shape), int(s), int(start), int(end),
                             out.element_size(), 1, _stream(stream)), "tvc_slab_copy")
    return out


def split_tensor(A: torch.Tensor, s: int, starts, *, shape=None, stream=None) -> list:
    """The ranks' dense subtensors of A cut along s at `starts`."""
    return [slab_extract(A, s, starts[r], starts[r + 1], shape=shape, stream=stream) for r in range(len(starts) - 1)]


def _split_args(slabs, starts, shape):
    parts = len(starts) - 1
    if parts < 1 or len(slabs) != parts:
        raise ValueError("one slab per rank")
    code = dtype_code(slabs[0])
    if any(dtype_code(t) != code for t in slabs):
        raise ValueError("slabs differ in storage type")
    arr = (ctypes.c_int64 * (parts + 1))(*[int(v) for v in starts])
    ptrs = (ctypes.c_void_p * parts)(*[t.data_ptr() for t in slabs])
    return parts, code, arr, ptrs


def dtvc_workspace_size(starts, shape, s: int, mode: int, code: int) -> int:
    lib = load_library()
    parts = len(starts) - 1
    arr = (ctypes.c_int64 * (parts + 1))(*[int(v) for v in starts])
    return int(lib.dtvc_workspace_size(parts, arr, len(shape), _dims_array(shape), int(s), int(mode), int(code)))


def dtvc(slabs, starts, shape, s: int, mode: int, x: torch.Tensor, *, y=None, scales: torch.Tensor | None = None,
         alpha: float = 1.0, beta: float = 0.0, workspace: torch.Tensor | None = None, stream=None):
    """Distributed TVC over virtual ranks (Eq. 1 / Eq. 2).  slabs[r] is rank
    r's subtensor of the global tensor `shape` cut along s at `starts`.
    mode != s: returns the list of the ranks' output slabs; mode == s:
    returns the summed full-size output."""
    lib = load_library()
    shape = tuple(int(n) for n in shape)
    parts, code, arr, ptrs = _split_args(slabs, starts, shape)
    code = _with_vectors(code, x)
    vt = vec_dtype(code)
    if x.dtype != vt or x.numel() != shape[mode]:
        raise ValueError(f"x must be {vt} with {shape[mode]} entries")
    dev = slabs[0].device
    if mode == s:
        out_shape = tuple(n for i, n in enumerate(shape) if i != mode)
        if y is None:
            if beta != 0.0:
                raise ValueError("beta != 0 needs y")
            y = torch.empty(out_shape, dtype=vt, device=dev)
        outs = [y]
    else:
        if y is None:
            if beta != 0.0:
                raise ValueError("beta != 0 needs y")
            outs = []
            for r in range(parts):
                sh = _slab_shape(shape, s, starts[r], starts[r + 1])
                outs.append(torch.empty(tuple(n for i, n in enumerate(sh) if i != mode), dtype=vt, device=dev))
        else:
            outs = list(y)
    _check_cuda(x, scales, workspace, *slabs, *outs)
    if workspace is None:
        need = lib.dtvc_workspace_size(parts, arr, len(shape), _dims_array(shape), int(s), int(mode), code)
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    yp = (ctypes.c_void_p * len(outs))(*[t.data_ptr() for t in outs])
    _check(lib.dtvc(ptrs, parts, arr, len(shape), _dims_array(shape), int(s), int(mode), _ptr(x), yp, code,
                    _ptr(scales), float(alpha), float(beta), _ptr(workspace), workspace.numel(), _stream(stream)),
           "dtvc")
    return outs[0] if mode == s else outs


def dhopm_workspace_size(starts, shape, s: int, code: int) -> int:
    lib = load_library()
    parts = len(starts) - 1
    arr = (ctypes.c_int64 * (parts + 1))(*[int(v) for v in starts])
    return int(lib.dhopm_workspace_size(parts, arr, len(shape), _dims_array(shape), int(s), int(code)))


def dhopm(slabs, starts, shape, s: int, xs, iters: int, tol: float = 0.0, *, scales: torch.Tensor | None = None,
          workspace: torch.Tensor | None = None, stream=None, inplace: bool = False) -> HopmResult:
    """Distributed three-buffer HOPM (Algorithm 1) over virtual ranks: the
    ranks' slabs cut along s at `starts`, global start vectors xs."""
    lib = load_library()
    shape = tuple(int(n) for n in shape)
    if len(shape) < 2 or len(xs) != len(shape):
        raise ValueError("dhopm needs order >= 2 and one start vector per mode")
    parts, code, arr, ptrs = _split_args(slabs, starts, shape)
    code = _with_vectors(code, xs[-1])
    vt = vec_dtype(code)
    xs = [v if inplace else v.clone() for v in xs]
    for m, v in enumerate(xs):
        if v.dtype != vt or v.numel() != shape[m]:
            raise ValueError(f"x[{m}] must be {vt} with {shape[m]} entries")
    _check_cuda(scales, workspace, *slabs, *xs)
    dev = slabs[0].device
    lam = torch.zeros(1, dtype=torch.float64, device=dev)
    sweeps = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    hist = torch.zeros(max(1, iters), dtype=torch.float64, device=dev)
    dims = _dims_array(shape)
    if workspace is None:
        need = lib.dhopm_workspace_size(parts, arr, len(shape), dims, int(s), code)
        workspace = torch.empty(max(1, need), dtype=torch.uint8, device=dev)
    xp = (ctypes.c_void_p * len(xs))(*[v.data_ptr() for v in xs])
    _check(lib.dhopm(ptrs, parts, arr, len(shape), dims, int(s), xp, int(iters), float(tol), _ptr(lam), _ptr(sweeps),
                     _ptr(status), _ptr(hist), code, _ptr(scales), _ptr(workspace), workspace.numel(),
                     _stream(stream)), "dhopm")
    return HopmResult(xs, lam, sweeps, status, hist)
