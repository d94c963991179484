"""GPU parity of the power method (through the C ABI) and of the per-slab
quantiser, against the FP64 oracle.

Tolerances: FP64 lambda history 1e-12 relative, x_j within 1e-10; FP32
storage 1e-5; narrow storage: kernel against the oracle on the same codes
1e-5 (FP32 accumulation), lambda against the FP64 oracle on the unquantised
values within 1e-3 for BF16 and binary16 (E4M3: see
LAMBDA_STORAGE_BOUND_256; the full-size workload holds every format to
1e-3).  Quantiser codes bit-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

VEC = {oracle.F64: torch.float64, oracle.F32: torch.float32, oracle.BF16: torch.float32,
       oracle.E4M3: torch.float32, oracle.F16: torch.float32}


def ones_start(dims, code):
    return [torch.full((n,), 1.0 / math.sqrt(n), dtype=VEC[code], device=gu.DEV) for n in dims]


def ones_np(dims):
    return [np.ones(n) / math.sqrt(n) for n in dims]


def as_stored(xs, code):
    """Vectors as the GPU holds them: FP64, or rounded to binary32."""
    if code == oracle.F64:
        return [np.asarray(v, dtype=np.float64).copy() for v in xs]
    return [np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64) for v in xs]


def to_dev_vectors(xs, code):
    return [torch.from_numpy(np.asarray(v, dtype=np.float64)).to(dtype=VEC[code], device=gu.DEV) for v in xs]


def run_gpu(A, dims, code, iters, tol=0.0, scales=None, xs=None):
    r = tg.hopm(gu.to_dev(A), xs if xs is not None else ones_start(dims, code), iters, tol,
                scales=gu.to_dev(scales) if scales is not None else None, shape=dims)
    torch.cuda.synchronize()
    return r


def check_against(r, ref, code):
    tol = 1e-12 if code == oracle.F64 else 1e-5
    n = ref["sweeps"]
    assert int(r.sweeps.item()) == n
    hist = r.lam_hist.cpu().numpy()[:n]
    np.testing.assert_allclose(hist, ref["lam_hist"], rtol=tol)
    assert abs(r.lam.item() - ref["lam"]) <= tol * ref["lam"]
    xtol = 1e-10 if code == oracle.F64 else 2e-4
    for xg, xr in zip(r.x, ref["x"]):
        assert np.max(np.abs(xg.cpu().numpy().astype(np.float64) - xr)) <= xtol


SHAPES = [(9, 7), (5, 6, 7), (4, 5, 3, 6), (3, 4, 2, 3, 5), (2, 3, 2, 2, 3, 2), (40, 33, 70), (130, 64),
          (3, 200, 2), (17, 1, 9)]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16], ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_hopm_matches_oracle(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    iters = 8
    ref = oracle.hopm(Ao, ones_np(dims), iters, scales=scales)
    assert ref["status"] == 0
    r = run_gpu(A, dims, code, iters, scales=scales)
    assert int(r.status.item()) == 0
    check_against(r, ref, code)


def test_config_128cube_fp64_20_sweeps():
    """Plain-method workload: 128^3 FP64 uniform[-1,1] seed 0, 20 sweeps from
    normalised all-ones vectors."""
    dims = (128, 128, 128)
    A = synth.tensor("u64", 0, dims)
    ref = oracle.hopm(A, ones_np(dims), 20)
    r = run_gpu(A, dims, oracle.F64, 20)
    check_against(r, ref, oracle.F64)
    # the three-buffer oracle agrees as well
    ref3 = oracle.hopm3(A, ones_np(dims), 20)
    np.testing.assert_allclose(r.lam_hist.cpu().numpy(), ref3["lam_hist"], rtol=1e-12)


@pytest.mark.parametrize("code", [oracle.F64, oracle.F32])
def test_rank1_converges_in_one_sweep(code):
    dims = (6, 5, 7, 4)
    us = [synth.vector("u64", 3, 60 + j, n) for j, n in enumerate(dims)]
    A = np.einsum("i,j,k,l->ijkl", *us)
    if code == oracle.F32:
        A = A.astype(np.float32)
    r = run_gpu(A, dims, code, 1)
    lam_true = np.prod([np.linalg.norm(u) for u in us])
    tol = 1e-12 if code == oracle.F64 else 1e-5
    assert abs(r.lam.item() - lam_true) <= tol * lam_true
    for xg, u in zip(r.x, us):
        assert abs(abs(np.dot(xg.cpu().numpy(), u / np.linalg.norm(u))) - 1.0) <= 10 * tol


def test_matrix_top_singular_value():
    A = synth.tensor("u64", 5, (50, 30))
    r = run_gpu(A, A.shape, oracle.F64, 400, tol=1e-15)
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(r.lam.item() - s[0]) <= 1e-10 * s[0]


def test_stopping_rule_and_unused_x0():
    dims = (7, 6, 5)
    A = synth.tensor("u64", 1, dims)
    ref = oracle.hopm(A, ones_np(dims), 500, tol=1e-7)
    assert ref["sweeps"] < 500
    r = run_gpu(A, dims, oracle.F64, 500, tol=1e-7)
    check_against(r, ref, oracle.F64)
    xs = ones_start(dims, oracle.F64)
    xs[0] = torch.full_like(xs[0], 123.0)
    r2 = run_gpu(A, dims, oracle.F64, 6, xs=xs)
    r1 = run_gpu(A, dims, oracle.F64, 6)
    assert torch.equal(r1.lam_hist, r2.lam_hist)


def test_zero_and_nonfinite_status():
    A = np.zeros((4, 5, 3))
    r = run_gpu(A, A.shape, oracle.F64, 3)
    assert int(r.status.item()) == 5
    assert int(r.sweeps.item()) == 0
    B = synth.tensor("u64", 2, (4, 5, 3))
    B[1, 2, 0] = np.nan
    r = run_gpu(B, B.shape, oracle.F64, 3)
    assert int(r.status.item()) == 6
    with pytest.raises(tg.TVCError):
        r.check()


def test_hopm_deterministic():
    dims = (30, 40, 50)
    A = synth.tensor("u64", 4, dims)
    a = run_gpu(A, dims, oracle.F64, 5)
    b = run_gpu(A, dims, oracle.F64, 5)
    assert torch.equal(a.lam_hist, b.lam_hist)
    for xa, xb in zip(a.x, b.x):
        assert torch.equal(xa, xb)


@pytest.mark.parametrize("dims", [(5, 40, 33), (3, 1, 100), (7,), (2, 3, 4, 5)], ids=lambda d: "x".join(map(str, d)))
def test_quantise_bit_exact(dims):
    src = synth.tensor("lognormal", 3, dims).astype(np.float32)
    src.ravel()[::97] = 0.0
    for code in (oracle.BF16, oracle.E4M3, oracle.F16):
        for trunc in ((False, True) if code == oracle.BF16 else (False,)):
            c_ref, s_ref = oracle.quantise(src, code, truncate=trunc)
            codes, scales, status = tg.quantise(gu.to_dev(src), code, truncate=trunc)
            assert int(status.item()) == 0
            assert np.array_equal(scales.cpu().numpy(), s_ref)
            got = codes.cpu().numpy()
            if code == oracle.F16:  # compare the binary16 bits
                got, c_ref = got.view(np.uint16), c_ref.view(np.uint16)
            assert np.array_equal(got, c_ref)


def test_quantise_nonfinite_status_and_zero_slab():
    src = synth.tensor("lognormal", 1, (3, 8, 8)).astype(np.float32)
    src[1] = 0.0
    codes, scales, status = tg.quantise(gu.to_dev(src), tg.E4M3)
    assert int(status.item()) == 0 and scales[1].item() == 1.0 and int(codes[1].abs().sum().item()) == 0
    src[2, 3, 3] = np.inf
    _, _, status = tg.quantise(gu.to_dev(src), tg.E4M3)
    assert int(status.item()) == 6
    # binary16: overflow (and NaN) give non-finite codes and set the status;
    # every code is still written and equals the oracle's
    src = synth.tensor("lognormal", 1, (3, 8, 8)).astype(np.float32)
    src[0, 1, 2] = 7e4
    src[1, 2, 3] = np.nan
    codes, scales, status = tg.quantise(gu.to_dev(src), tg.F16)
    assert int(status.item()) == 6
    ref, _ = oracle.quantise(src, oracle.F16, allow_nonfinite=True)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), ref.view(np.uint16))


# Storage error of lambda at this reduced size, against the FP64 oracle on
# the binary32 source.  BF16 and binary16 meet the 1e-3 target of the
# full-size 2048^3 workload here already (1.6e-4, 1.6e-5).  E4M3 rounds each
# element with a relative RMS error of 2.6%; its first-order effect on lambda,
# E(x_0, x_1, x_2) for the rounding error tensor E, shrinks like 1/sqrt(n)
# with the side n: 1.5e-3 at 256^3 and 3.7e-4 at 2048^3, where
# test_fullsize_hopm_gpu.py asserts the 1e-3 target.  Here E4M3 is held to
# 2e-3.
LAMBDA_STORAGE_BOUND_256 = {oracle.BF16: 1e-3, oracle.E4M3: 2e-3, oracle.F16: 1e-3}


@pytest.mark.parametrize("code", [oracle.BF16, oracle.E4M3, oracle.F16], ids=["bf16", "e4m3", "f16"])
def test_low_precision_hopm_lambda_vs_fp64(code):
    """Mixed-precision recipe at reduced size (256^3): N(0,1)exp(U[-3,3])
    entries, stored narrow with per-slab scales, 30 sweeps.  The GPU's codes
    equal the oracle quantiser's; lambda against the oracle on those codes
    (kernel error, 1e-5) and on the binary32 source (storage error)."""
    dims = (256, 256, 256)
    src = synth.tensor("lognormal", 0, dims).astype(np.float32)
    codes_o, scales_o = oracle.quantise(src, code)
    codes, scales, status = tg.quantise(gu.to_dev(src), code)
    assert int(status.item()) == 0
    got_codes = codes.cpu().numpy()
    if code == oracle.F16:
        got_codes, codes_cmp = got_codes.view(np.uint16), codes_o.view(np.uint16)
    else:
        codes_cmp = codes_o
    assert np.array_equal(got_codes.reshape(codes_cmp.shape), codes_cmp)
    assert np.array_equal(scales.cpu().numpy(), scales_o)
    r = tg.hopm(codes, ones_start(dims, code), 30, scales=scales, shape=dims)
    torch.cuda.synchronize()
    ref = oracle.hopm(src, ones_np(dims), 30)
    err = abs(r.lam.item() - ref["lam"]) / ref["lam"]
    print(f"{ {oracle.BF16: 'bf16', oracle.E4M3: 'e4m3', oracle.F16: 'f16'}[code]} lambda rel err vs FP64 oracle: {err:.3e}")
    assert err <= LAMBDA_STORAGE_BOUND_256[code]
    # kernel error: the oracle on the same stored codes (its own quantiser's)
    ref_q = oracle.hopm(codes_o, ones_np(dims), 30, scales=scales_o)
    assert abs(r.lam.item() - ref_q["lam"]) <= 1e-5 * ref_q["lam"]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_hopm_single_double(dims):
    """binary32 storage with FP64 vectors: the FP64 tolerances of the oracle's
    FP32 path (which promotes every element to FP64)."""
    A = synth.tensor("u32", 0, dims)
    ref = oracle.hopm(A, ones_np(dims), 8)
    r = tg.hopm(gu.to_dev(A), ones_start(dims, oracle.F64), 8, shape=dims)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    check_against(r, ref, oracle.F64)


# ------------------------------------------------------------ Jacobi HOPM

@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16],
                         ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_hopm_jacobi_matches_oracle(dims, code):
    """Sweep by sweep: the oracle iterates from all-ones on its own vectors;
    before each sweep both sides start from the oracle's current vectors (as
    the GPU stores them: binary32 for the FP32-vector types), and one GPU
    sweep is compared with one oracle sweep.  (A Jacobi iteration need not
    contract, so differences of rounding may grow over many sweeps; the map
    itself is what must agree.)"""
    A, Ao, scales = gu.inputs(dims, code)
    st = gu.to_dev(scales) if scales is not None else None
    xs_o = ones_np(dims)
    for t in range(5):
        start = as_stored(xs_o, code)
        ref = oracle.hopm_jacobi(Ao, start, 1, scales=scales)
        assert ref["status"] == 0
        r = tg.hopm_jacobi(gu.to_dev(A), to_dev_vectors(start, code), 1, scales=st, shape=dims)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        check_against(r, ref, code)
        xs_o = ref["x"]


def test_hopm_jacobi_single_double_and_stopping_rule():
    # a dominant rank-1 term (the planted workload's structure), where the
    # Jacobi iteration converges; binary32 storage with FP64 vectors
    dims = (9, 8, 7)
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    A = synth.tensor("planted", 0, dims, us=us).astype(np.float32)
    ref = oracle.hopm_jacobi(A, ones_np(dims), 200, 1e-10)
    r = tg.hopm_jacobi(gu.to_dev(A), ones_start(dims, oracle.F64), 200, 1e-10, shape=dims)
    torch.cuda.synchronize()
    check_against(r, ref, oracle.F64)
    assert int(r.sweeps.item()) == ref["sweeps"] < 200


# last dimensions that are multiples of 32 x (16 bytes of codes): the
# single-pass kernel (T = A x_{d-1} x_{d-1} and z_{d-1} = A^T w from one read
# of A) with 1, 2, 4 and 8 warps per row, slab scales applied in the kernel
# (one warp per row) or after it, a single row, and ragged row counts
SINGLE_PASS_SHAPES = [(6, 5, 256), (7, 3, 512), (3, 1024), (2, 3, 2048), (1, 4096), (5, 4, 3, 128)]


@pytest.mark.parametrize("dims", SINGLE_PASS_SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", [oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16],
                         ids=["f32", "bf16", "e4m3", "f16"])
def test_hopm_jacobi_single_pass_kernel(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    st = gu.to_dev(scales) if scales is not None else None
    xs_o = ones_np(dims)
    for t in range(3):
        start = as_stored(xs_o, code)
        ref = oracle.hopm_jacobi(Ao, start, 1, scales=scales)
        r = tg.hopm_jacobi(gu.to_dev(A), to_dev_vectors(start, code), 1, scales=st, shape=dims)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        check_against(r, ref, code)
        xs_o = ref["x"]


def test_read_status_after_a_zero_tensor():
    """The status word of a power method on a zero tensor, read through the
    C ABI once the queued work is done: TVC_ERR_ZERO_NORM."""
    dims = (3, 4, 5)
    A = torch.zeros(dims, dtype=torch.float64, device=gu.DEV)
    xs = [torch.full((n,), 1.0 / math.sqrt(n), dtype=torch.float64, device=gu.DEV) for n in dims]
    r = tg.hopm(A, xs, 3)
    assert tg.read_status(r.status) == 5
    ok = torch.zeros(1, dtype=torch.int32, device=gu.DEV)
    assert tg.read_status(ok) == 0
