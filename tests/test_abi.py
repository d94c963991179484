"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument validation answers without a GPU (nothing is launched)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT

LIB = os.path.join(ROOT, "paper_2501_03121_gb300", "_lib", "libtvc_gb300.so")


def _build():
    from paper_2501_03121_gb300 import build as b
    return b.build()


@pytest.fixture(scope="module")
def lib():
    _build()
    return ctypes.CDLL(LIB)


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**\s*([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("tvc", "tvc_ex", "tvc_workspace_size", "tvc_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.tvc_status_string.restype = ctypes.c_char_p
    for s in range(8):
        assert lib.tvc_status_string(s).startswith(b"TVC_")
    assert b"unknown" in lib.tvc_status_string(99)


def test_validation_without_gpu(lib):
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.tvc.argtypes = [P, I, P, I, P, P, I, P]
    lib.tvc.restype = I
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    fake = ctypes.c_void_p(1 << 20)
    assert lib.tvc(None, 3, dims, 1, fake, fake, 0, None) == 1          # null A
    assert lib.tvc(fake, 3, dims, 3, fake, fake, 0, None) == 1          # mode out of range
    assert lib.tvc(fake, 0, dims, 0, fake, fake, 0, None) == 1          # order 0
    assert lib.tvc(fake, 17, dims, 0, fake, fake, 0, None) == 1         # order > 16
    assert lib.tvc(fake, 3, dims, 1, fake, fake, 9, None) == 1          # dtype
    bad = (ctypes.c_int64 * 3)(4, 0, 6)
    assert lib.tvc(fake, 3, bad, 1, fake, fake, 0, None) == 1           # zero size
    huge = (ctypes.c_int64 * 3)(1 << 30, 1 << 30, 1 << 30)
    assert lib.tvc(fake, 3, huge, 1, fake, fake, 0, None) == 1          # N >= 2^62
    mis = ctypes.c_void_p((1 << 20) + 4)
    assert lib.tvc(mis, 3, dims, 1, fake, fake, 0, None) == 1           # A not 8-byte aligned (FP64)


def test_workspace_size_query(lib):
    lib.tvc_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.tvc_workspace_size.restype = ctypes.c_size_t
    dims = (ctypes.c_int64 * 2)(65536, 16384)
    # FP64 always needs the split x; a short-output contraction also needs partials.
    assert lib.tvc_workspace_size(2, dims, 0, 0) >= 65536 * 8 + 16384 * 8
    assert lib.tvc_workspace_size(2, dims, 1, 1) == 0 or lib.tvc_workspace_size(2, dims, 1, 1) > 0
    bad = (ctypes.c_int64 * 2)(0, 3)
    assert lib.tvc_workspace_size(2, bad, 0, 0) == 0


def _align256(n):
    return (n + 255) // 256 * 256


def test_workspace_of_fp64_row_plans(lib):
    """Host planning of FP64 rows, through the workspace query (no GPU):
    rows of odd length >= 1024 read 16-byte pairs against a second, shifted
    copy of the split x (n_k + 2 entries); rows whose split x outgrows L1
    (n_k * 8 > 160 KB) run in segments of about 4096 entries with their
    partial sums in the workspace, unless those would pass 16 MB."""
    lib.tvc_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.tvc_workspace_size.restype = ctypes.c_size_t
    F64 = 0
    xs = lambda nk: _align256(nk * 8)  # noqa: E731  the split x (two floats per entry)
    # odd rows of 4097 elements, 100000 rows (no split of n_k): split x and its shifted copy
    odd = (ctypes.c_int64 * 2)(100000, 4097)
    assert lib.tvc_workspace_size(2, odd, 1, F64) == xs(4097) + _align256(4099 * 8)
    even = (ctypes.c_int64 * 2)(100000, 4096)
    assert lib.tvc_workspace_size(2, even, 1, F64) == xs(4096)
    # 30623 x 30623 mode 1: 8 segments of the rows, partials 8 x 30623 doubles
    t1 = (ctypes.c_int64 * 2)(30623, 30623)
    got = lib.tvc_workspace_size(2, t1, 1, F64)
    assert got == xs(30623) + _align256((30623 + 2) * 8) + _align256(8 * 30623 * 8)
    # a million such rows: 8 segments would need 64 MB of partials, so no segments
    big = (ctypes.c_int64 * 2)(1000000, 30623)
    assert lib.tvc_workspace_size(2, big, 1, F64) == xs(30623) + _align256((30623 + 2) * 8)


def test_tmc_validation_without_gpu(lib):
    P, I, D, Z, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_int64
    lib.tmc.argtypes = [P, I, P, I, P, L, P, I, P, D, D, P, Z, P]
    lib.tmc.restype = I
    lib.tmc_workspace_size.argtypes = [I, P, I, L, I]
    lib.tmc_workspace_size.restype = Z
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    fake = ctypes.c_void_p(1 << 20)
    args = lambda A=fake, X=fake, Y=fake, R=3, dt=0, mode=1, d=dims: (A, 3, d, mode, X, R, Y, dt, None, 1.0, 0.0,
                                                                        None, 0, None)
    assert lib.tmc(*args(R=0)) == 1                                  # R < 1
    assert lib.tmc(*args(A=None)) == 1                               # null A
    assert lib.tmc(*args(X=None)) == 1                               # null X
    assert lib.tmc(*args(mode=3)) == 1                               # mode out of range
    assert lib.tmc(*args(dt=9)) == 1                                 # dtype
    assert lib.tmc(*args(Y=ctypes.c_void_p((1 << 20) + 4))) == 1     # Y not 8-byte aligned (FP64 vectors)
    long = (ctypes.c_int64 * 2)(2, 1 << 20)
    need = lib.tmc_workspace_size(2, long, 1, 8, 1)                  # two outputs per row of X: split n_k
    assert need > 0
    assert lib.tmc(fake, 2, long, 1, fake, 8, fake, 1, None, 1.0, 0.0, None, 0, None) == 3   # workspace
    assert lib.tmc_workspace_size(2, long, 1, 0, 1) == 0


def test_cpals_validation_without_gpu(lib):
    P, I, Z, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_int64
    lib.khatri_rao.argtypes = [P, I, P, L, P, I, P]
    lib.khatri_rao.restype = I
    lib.mttkrp.argtypes = [P, I, P, I, P, L, P, I, P, P, Z, P]
    lib.mttkrp.restype = I
    lib.mttkrp_workspace_size.argtypes = [I, P, I, L, I]
    lib.mttkrp_workspace_size.restype = Z
    fake = ctypes.c_void_p(1 << 20)
    mats = (ctypes.c_void_p * 2)(1 << 20, 1 << 21)
    rows = (ctypes.c_int64 * 2)(3, 4)
    assert lib.khatri_rao(mats, 0, rows, 2, fake, 0, None) == 1        # no matrices
    assert lib.khatri_rao(mats, 2, rows, 0, fake, 0, None) == 1        # R < 1
    assert lib.khatri_rao(mats, 2, rows, 2, fake, 2, None) == 1        # matrices are FP64 or FP32
    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    facs = (ctypes.c_void_p * 3)(1 << 20, 0, 1 << 21)
    assert lib.mttkrp(fake, 3, dims, 1, facs, 0, fake, 1, None, fake, 1 << 30, None) == 1   # R < 1
    assert lib.mttkrp(fake, 3, dims, 0, facs, 2, fake, 1, None, fake, 1 << 30, None) == 1   # factor 1 missing
    assert lib.mttkrp(fake, 3, dims, 1, facs, 2, fake, 1, None, None, 0, None) == 3         # no workspace
    need = lib.mttkrp_workspace_size(3, dims, 1, 2, 1)
    assert need >= (2 * 6 + 2 * 4 + 2 * 5 * 4) * 4                      # Khatri-Rao rows and the intermediate
    assert lib.mttkrp_workspace_size(3, dims, 3, 2, 1) == 0              # bad mode


def _mttkrp_ws_expected(lib, dims, k, R, code):
    """The MTTKRP workspace from the plan's rules: the larger side of mode k
    is contracted by the pass over A; for the modes after k, only the
    longest trailing block whose transposed Khatri-Rao rows fit 16 MB."""
    import math
    vs = 8 if code in (0, 5) else 4
    d = len(dims)
    u, nk, v, n0 = math.prod(dims[:k]), dims[k], math.prod(dims[k + 1:]), dims[0]
    right = v >= u
    va = vb = 1
    if right:
        msplit, vb = k + 1, v
        while msplit < d - 1 and R * vb * vs > (16 << 20):
            vb //= dims[msplit]
            msplit += 1
        va = v // vb
        view, mode = ((nk * va, vb), 1) if k == 0 else ((n0, u * nk * va // n0, vb), 2)
        t_is_m = k == 0 and va == 1
    else:
        view, mode, t_is_m = (u, nk * v), 0, False
    kt = R * (vb if right else u)
    kw = R * (u * va if right else v)
    t = 0 if t_is_m else R * nk * (u * va if right else v)
    vd = (ctypes.c_int64 * len(view))(*view)
    tmc_ws = lib.tmc_workspace_size(len(view), vd, mode, R, code)
    up = lambda x: (x + 255) // 256 * 256  # noqa: E731
    off_kw = up(kt * vs)
    off_t = up(off_kw + kw * vs)
    off_tmc = up(off_t + t * vs)
    return off_tmc + tmc_ws


def test_mttkrp_plan_workspace_without_gpu(lib):
    lib.mttkrp_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    lib.mttkrp_workspace_size.restype = ctypes.c_size_t
    lib.tmc_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    lib.tmc_workspace_size.restype = ctypes.c_size_t
    cases = [((3, 4, 5), 1, 3, 1), ((40, 3, 6), 2, 8, 0), ((6, 3, 40), 0, 8, 2), ((4, 96, 96, 96), 0, 8, 1),
             ((4, 96, 96, 96), 1, 8, 0), ((2, 5, 128, 8192), 1, 8, 1), ((1024, 1024, 1024), 2, 16, 1),
             ((256, 256, 256, 256), 0, 8, 1), ((7,), 0, 4, 1)]
    for dims, k, R, code in cases:
        arr = (ctypes.c_int64 * len(dims))(*dims)
        got = lib.mttkrp_workspace_size(len(dims), arr, k, R, code)
        assert got == _mttkrp_ws_expected(lib, dims, k, R, code), (dims, k, R, code)


def test_read_status_validation_without_gpu(lib):
    lib.tvc_read_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.tvc_read_status.restype = ctypes.c_int
    out = ctypes.c_int(0)
    assert lib.tvc_read_status(None, ctypes.byref(out), None) == 1
    assert lib.tvc_read_status(ctypes.c_void_p(1 << 20), None, None) == 1
