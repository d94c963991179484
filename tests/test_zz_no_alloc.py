"""tvc_noalloc, the contraction entry point for callers that cannot allocate
device memory: plug-ins whose host framework owns all device memory through
its own pool, and deployments that forbid device allocation after start-up.
It must give the results of tvc() and of the FP64 oracle, within the
tolerances of the other tests, call after call on its one shared scratch
array; refuse contractions whose scratch would not fit; and, once loaded,
leave the device's free memory unchanged however often it is called.

This file is named so that pytest collects it last; it also passes alone in
a fresh process.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

TOL = {tg.F64: 1e-12, tg.F32: 1e-5}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_noalloc_matches_tvc_and_oracle_two_calls_in_a_row():
    lib = tg.load_library()
    for shape, mode, code in CASES:
        kind = "u64" if code == tg.F64 else "u32"
        Ah = synth.tensor(kind, 7, shape)
        xh = synth.vector(kind, 8, 1 + mode, shape[mode])
        A, x = gu.to_dev(Ah), gu.to_dev(xh)
        ref = tg.tvc(A, mode, x).cpu().numpy()
        ref_oracle = oracle.tvc(Ah, mode, xh)
        for _ in range(2):
            y = torch.full(ref.shape, float("nan"), dtype=x.dtype, device=gu.DEV)
            assert _noalloc(lib, A, shape, mode, x, y, code) == 0
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert gu.rel_l2(got, ref) <= TOL[code], (shape, mode)
            assert gu.rel_l2(got, ref_oracle) <= TOL[code], (shape, mode)


def test_noalloc_narrow_storage_with_scales():
    lib = tg.load_library()
    shape = (8, 300, 70)
    src = synth.tensor("lognormal", 2, shape).astype(np.float32)
    codes_h, scales_h = oracle.quantise(src, oracle.E4M3)
    codes, scales = gu.to_dev(codes_h), gu.to_dev(scales_h)
    for mode in range(3):
        xh = synth.vector("u32", 3, 1 + mode, shape[mode])
        x = gu.to_dev(xh)
        ref = tg.tvc(codes, mode, x, scales=scales, shape=shape).cpu().numpy()
        ref_oracle = oracle.tvc(codes_h, mode, xh, scales=scales_h)
        y = torch.empty(ref.shape, dtype=torch.float32, device=gu.DEV)
        assert _noalloc(lib, codes, shape, mode, x, y, tg.E4M3, scales) == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert gu.rel_l2(got, ref) <= 1e-5
        assert gu.rel_l2(got, ref_oracle) <= 1e-5


def test_noalloc_refuses_oversize_scratch():
    lib = tg.load_library()
    n = (1 << 23) + 5  # order 1, FP64: the split x alone needs 64 MiB
    A = torch.zeros(n, dtype=torch.float64, device=gu.DEV)
    x = torch.zeros(n, dtype=torch.float64, device=gu.DEV)
    y = torch.zeros(1, dtype=torch.float64, device=gu.DEV)
    assert _noalloc(lib, A, (n,), 0, x, y, tg.F64) == 3  # TVC_ERR_WORKSPACE
    # invalid arguments are still caught first
    assert _noalloc(lib, A, (n,), 1, x, y, tg.F64) == 1


# Run in a fresh process with every module loaded at context creation, so
# that nothing is loaded (and allocated) lazily by a later first launch.
_NO_ALLOC_CHILD = textwrap.dedent("""
    import ctypes, sys
    import torch
    sys.path.insert(0, {root!r})
    import paper_2501_03121_gb300 as tg
    lib = tg.load_library()
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.tvc_noalloc.argtypes = [P, I, P, I, P, P, I, P, P]
    lib.tvc_noalloc.restype = I
    dev = torch.device("cuda:0")
    cases = {cases!r}
    bufs = []
    for shape, mode, code in cases:
        dt = torch.float64 if code == tg.F64 else torch.float32
        n = 1
        for d in shape:
            n *= d
        A = torch.rand(n, dtype=dt, device=dev)
        x = torch.rand(shape[mode], dtype=dt, device=dev)
        y = torch.empty(n // shape[mode], dtype=dt, device=dev)
        bufs.append((shape, mode, code, A, x, y))
    def call(shape, mode, code, A, x, y):
        dims = (ctypes.c_int64 * len(shape))(*shape)
        st = lib.tvc_noalloc(P(A.data_ptr()), len(shape), dims, mode, P(x.data_ptr()), P(y.data_ptr()), code,
                             None, P(torch.cuda.current_stream().cuda_stream))
        assert st == 0, st
    call(*bufs[0])  # first call: looks up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for b in bufs:
            call(*b)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print("free bytes before", free0, "after", free1)
    assert free1 == free0, (free0, free1)
    print("NO_ALLOC_OK")
""")


def test_noalloc_allocates_no_device_memory():
    code = _NO_ALLOC_CHILD.format(root=ROOT, cases=CASES)
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "NO_ALLOC_OK" in r.stdout, r.stdout + r.stderr
