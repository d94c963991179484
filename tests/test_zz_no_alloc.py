"""tvc_noalloc, the contraction entry point for callers that cannot allocate
device memory (host callbacks where CUDA calls are not allowed, plug-ins
whose framework owns all device memory, deployments that forbid allocation
after start-up).  It must give the same results as tvc(), within the
tolerances of the other tests, call after call on its one shared scratch
array, and refuse contractions whose scratch would not fit.

This file is named so that pytest collects it last; it also passes alone in
a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

TOL = {tg.F64: 1e-12, tg.F32: 1e-5}


def _noalloc(lib, A, shape, mode, x, y, code, scales=None):
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.tvc_noalloc.argtypes = [P, I, P, I, P, P, I, P, P]
    lib.tvc_noalloc.restype = I
    dims = (ctypes.c_int64 * len(shape))(*shape)
    st = lib.tvc_noalloc(P(A.data_ptr()), len(shape), dims, mode, P(x.data_ptr()), P(y.data_ptr()), code,
                         P(scales.data_ptr()) if scales is not None else None,
                         P(torch.cuda.current_stream().cuda_stream))
    return st


# Cases that use the scratch: FP64 always stores the split x there, and
# these shapes also split n_k and keep partial sums there.
CASES = [((20000, 64), 0, tg.F64), ((3, 300000), 1, tg.F32), ((2, 5000, 9), 1, tg.F64), ((6, 70, 33), 2, tg.F64),
         ((65536, 256), 0, tg.F32)]


def test_noalloc_matches_tvc_two_calls_in_a_row():
    lib = tg.load_library()
    for shape, mode, code in CASES:
        kind = "u64" if code == tg.F64 else "u32"
        A = gu.to_dev(synth.tensor(kind, 7, shape))
        x = gu.to_dev(synth.vector(kind, 8, 1 + mode, shape[mode]))
        ref = tg.tvc(A, mode, x)
        for _ in range(2):
            y = torch.full_like(ref, float("nan"))
            assert _noalloc(lib, A, shape, mode, x, y, code) == 0
            torch.cuda.synchronize()
            assert gu.rel_l2(y.cpu().numpy(), ref.cpu().numpy()) <= TOL[code], (shape, mode)


def test_noalloc_narrow_storage_with_scales():
    lib = tg.load_library()
    shape = (8, 300, 70)
    src = gu.to_dev(synth.tensor("lognormal", 2, shape).astype(np.float32))
    codes, scales, _ = tg.quantise(src, tg.E4M3)
    for mode in range(3):
        x = gu.to_dev(synth.vector("u32", 3, 1 + mode, shape[mode]))
        ref = tg.tvc(codes, mode, x, scales=scales)
        y = torch.empty_like(ref)
        assert _noalloc(lib, codes, shape, mode, x, y, tg.E4M3, scales) == 0
        torch.cuda.synchronize()
        assert gu.rel_l2(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


def test_noalloc_refuses_oversize_scratch():
    lib = tg.load_library()
    n = (1 << 23) + 5  # order 1, FP64: the split x alone needs 64 MiB
    A = torch.zeros(n, dtype=torch.float64, device=gu.DEV)
    x = torch.zeros(n, dtype=torch.float64, device=gu.DEV)
    y = torch.zeros(1, dtype=torch.float64, device=gu.DEV)
    assert _noalloc(lib, A, (n,), 0, x, y, tg.F64) == 3  # TVC_ERR_WORKSPACE
    # invalid arguments are still caught first
    assert _noalloc(lib, A, (n,), 1, x, y, tg.F64) == 1
