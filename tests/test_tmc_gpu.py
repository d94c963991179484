"""GPU parity of the mode-k tensor-matrix contraction (through the C ABI)
against the FP64 oracle: every mode and storage type, X with 1 to 21 rows
(one pass, several passes), split n_k, vector loads along rows and their
ragged tails, alpha/beta, exact gathers by selection matrices, integer
inputs bit for bit, and the 1024^3 workload sampled at full size.

FP64 values outside the float-float window are covered too.

Tolerances (relative l2 over the output): FP64 and single-double 1e-12,
FP32 and the narrow types (against the oracle on the same codes) 1e-5."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

# Reaching every kernel: column pieces (v > 1), rows by lane groups of 4 to
# 32 lanes (v == 1, rows of whole 16-byte pieces, an order-1 tensor with its
# per-entry slab scales), the generic kernel (ragged rows, FP64), split n_k
# (few outputs), several passes over A (R > 16) and ragged tails.
SHAPES = [(7,), (64,), (100003,), (5, 3), (4, 1), (3, 1, 5), (6, 5, 4, 3), (3, 50, 64), (5, 1000), (3, 4099),
          (4, 100, 7), (300, 40), (9, 33, 130), (7, 3072), (1001, 1536), (2, 3, 2, 3, 2, 3, 2), (3, 65536),
          (50, 256), (17, 48), (3, 7, 128), (2, 4096)]
CODES = [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16]
RS = [1, 3, 8, 13, 21]


def mat(code, R, n, sid, seed=2):
    if code == oracle.F64:
        return synth.tensor("u64", seed, (R, n), sid)
    return synth.tensor("u32", seed, (R, n), sid)


def gpu_tmc(A, k, X, scales=None, dims=None, **kw):
    st = gu.to_dev(scales) if scales is not None else None
    return tg.tmc(gu.to_dev(A), k, gu.to_dev(X), scales=st, shape=dims or A.shape, **kw).cpu().numpy()


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_tmc_every_mode(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    for k in range(len(dims)):
        for R in RS:
            X = mat(code, R, dims[k], synth.stream_x(k))
            ref = oracle.tmc(Ao, k, X, scales=scales)
            got = gpu_tmc(A, k, X, scales)
            assert got.shape == ref.shape
            assert gu.rel_l2(got, ref) <= gu.TOL[code], (dims, k, R)


@pytest.mark.parametrize("dims", [(5, 3), (3, 50, 64), (3, 4099), (1001, 1536), (6, 5, 4, 3), (3, 65536)],
                         ids=lambda d: "x".join(map(str, d)))
def test_tmc_single_double(dims):
    """binary32 storage, FP64 matrix and arithmetic."""
    A = synth.tensor("u32", 2, dims)
    for k in range(len(dims)):
        for R in (3, 8, 11):
            X = synth.tensor("u64", 3, (R, dims[k]), synth.stream_x(k))
            got = gpu_tmc(A, k, X)
            assert got.dtype == np.float64
            assert gu.rel_l2(got, oracle.tmc(A, k, X)) <= 1e-12, (dims, k, R)


@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_tmc_alpha_beta(code):
    dims = (6, 40, 33)
    A, Ao, scales = gu.inputs(dims, code)
    for k in range(3):
        X = mat(code, 5, dims[k], 60 + k)
        Y0 = mat(code, 1, 5 * (np.prod(dims) // dims[k]), 70 + k).reshape(
            tuple(5 if i == k else n for i, n in enumerate(dims)))
        Yt = gu.to_dev(Y0)
        tg.tmc(gu.to_dev(A), k, gu.to_dev(X), Y=Yt, scales=gu.to_dev(scales) if scales is not None else None,
               alpha=-0.75, beta=1.5, shape=dims)
        ref = oracle.tmc(Ao, k, X, scales=scales, Y=Y0, alpha=-0.75, beta=1.5)
        assert gu.rel_l2(Yt.cpu().numpy(), ref) <= gu.TOL[code], k


@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_tmc_selection_matrix_gathers_exactly(code):
    """Rows of X that pick one index of mode k: every output is one stored
    value (times its slab scale), exact for FP32 and the narrow types; FP64
    runs through the float-float split, whose low piece keeps 24 of the 29
    remaining bits, so each output is within 2^-47 of the value."""
    dims = (5, 24, 40)
    A, Ao, scales = gu.inputs(dims, code)
    deq = oracle.dequantise(Ao, scales) if scales is not None else Ao.astype(np.float64)
    vt = np.float64 if code == oracle.F64 else np.float32
    rng = np.random.default_rng(4)
    for k in range(3):
        for R in (dims[k], 9):
            pi = rng.permutation(dims[k])[:R] if R <= dims[k] else rng.integers(0, dims[k], size=R)
            X = np.zeros((R, dims[k]), dtype=vt)
            X[np.arange(R), pi] = 1.0
            got = gpu_tmc(A, k, X, scales)
            want = np.take(deq, pi, axis=k).astype(vt)
            if code == oracle.F64:
                assert np.all(np.abs(got - want) <= 2.0 ** -47 * np.abs(want)), (k, R)
            else:
                assert np.array_equal(got, want), (k, R)


@pytest.mark.parametrize("dims", [(7, 3072), (3, 65536), (9, 33, 130), (100003,)], ids=lambda d: "x".join(map(str, d)))
def test_tmc_integer_inputs_bit_exact_f64(dims):
    rng = np.random.default_rng(5)
    A = rng.integers(-8, 9, size=dims).astype(np.float64)
    for k in range(len(dims)):
        X = rng.integers(-8, 9, size=(10, dims[k])).astype(np.float64)
        assert np.array_equal(gpu_tmc(A, k, X), oracle.tmc(A, k, X)), k


@pytest.mark.parametrize("dims", [(9, 33, 130), (1001, 1536), (3, 65536), (40, 41, 5)],
                         ids=lambda d: "x".join(map(str, d)))
def test_tmc_fp64_values_outside_the_emulation_window(dims):
    """FP64 products run in float-float pieces on the FP32 pipe; zeros are
    exact and other elements or entries of X outside the pieces' window
    (huge, tiny, subnormal) send the thread to FP64 multiply-adds."""
    A = synth.tensor("u64", 4, dims)
    flat = A.ravel()
    rng = np.random.default_rng(6)
    pos = rng.choice(flat.size, size=min(600, flat.size), replace=False)
    flat[pos[:100]] = 0.0
    flat[pos[100:200]] *= 1e300
    flat[pos[200:300]] *= 1e-300
    flat[pos[300:400]] = 5e-324
    flat[pos[400:500]] *= 2.0 ** 70
    flat[pos[500:]] *= 2.0 ** -70
    for k in range(len(dims)):
        X = synth.tensor("u64", 1, (5, dims[k]), 1 + k)
        X[:, ::5] *= 1e-20
        X[:, 1::7] = 0.0
        assert gu.rel_l2(gpu_tmc(A, k, X), oracle.tmc(A, k, X)) <= 1e-12, (dims, k)
        X = synth.tensor("u64", 1, (5, dims[k]), 1 + k)
        assert gu.rel_l2(gpu_tmc(A, k, X), oracle.tmc(A, k, X)) <= 1e-12, (dims, k)
    A32 = synth.tensor("u32", 4, dims)
    f32 = A32.ravel()
    f32[pos[:100]] = 0.0
    f32[pos[100:200]] *= np.float32(1e30)
    f32[pos[200:300]] = np.float32(1e-42)
    for k in range(len(dims)):
        X = synth.tensor("u64", 1, (3, dims[k]), 1 + k)
        assert gu.rel_l2(gpu_tmc(A32, k, X), oracle.tmc(A32, k, X)) <= 1e-12, (dims, k)


def test_tmc_split_deterministic():
    dims = (2, 50000)
    A = gu.to_dev(synth.tensor("u32", 6, dims))
    X = gu.to_dev(synth.tensor("u32", 7, (6, 50000)))
    a = tg.tmc(A, 1, X)
    b = tg.tmc(A, 1, X)
    assert torch.equal(a, b)


def test_tmc_bad_arguments():
    A = gu.to_dev(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        tg.tmc(A, 1, gu.to_dev(np.zeros((2, 3))))
    with pytest.raises(ValueError):
        tg.tmc(A, 1, gu.to_dev(np.zeros((2, 4), dtype=np.float32)))
    with pytest.raises(ValueError):
        tg.tmc(A, 2, gu.to_dev(np.zeros((2, 4))))
    lib = tg.load_library()
    dims = tg._dims_array((3, 4))
    X = gu.to_dev(np.zeros((2, 4)))
    Y = gu.to_dev(np.zeros((3, 2)))
    assert lib.tmc(tg._ptr(A), 2, dims, 1, tg._ptr(X), 0, tg._ptr(Y), tg.F64, None, 1.0, 0.0, None, 0, None) != 0
    assert lib.tmc(tg._ptr(A), 2, dims, 1, tg._ptr(X), 2, tg._ptr(Y), 99, None, 1.0, 0.0, None, 0, None) != 0


@pytest.mark.slow
@pytest.mark.parametrize("code", [oracle.F64, oracle.F32], ids=["f64", "f32"])
def test_tmc_full_size_1024cube_sampled(code):
    """The 1024^3 workload with an 8-row matrix, every mode, outputs checked
    at sampled indices against the oracle from host-generated elements."""
    import synth.device as sd
    dims = (1024, 1024, 1024)
    kind = "u64" if code == oracle.F64 else "u32"
    dt = torch.float64 if code == oracle.F64 else torch.float32
    N = int(np.prod(dims, dtype=np.int64))
    At = torch.empty(N, dtype=dt, device=gu.DEV)
    sd.fill(At, kind, 0, synth.STREAM_A)
    rng = np.random.default_rng(1)
    R = 8
    for k in range(3):
        X = mat(code, R, dims[k], synth.stream_x(k), seed=1)
        Y = tg.tmc(At, k, gu.to_dev(X), shape=dims)
        Yr = Y.reshape(-1)
        picks, u, v = gu.sample_outputs(dims, k, 24, rng)
        for r in (0, 5, R - 1):
            i, l = picks // v, picks % v
            flat = (i * R + r) * v + l
            got = Yr[torch.from_numpy(flat).to(gu.DEV)].cpu().numpy()
            ref, mag = gu.oracle_at(kind, 0, dims, k, X[r], picks, v)
            assert gu.rel_l2(got, ref) <= gu.TOL[code], (k, r)
            assert np.all(np.abs(got - ref) <= 50 * gu.TOL[code] * mag), (k, r)
        del Y, Yr
    del At
    torch.cuda.empty_cache()


# BF16 storage with 8 <= R <= 64 and at least 152 tiles of 128 outputs goes
# to the tensor-core kernel (TMA tiles, tcgen05 MMAs on the three BF16 pieces
# of X, FP32 accumulation in tensor memory).  Last mode (K-major tiles):
# ragged n_k (zero filled to blocks of 64), ragged row tiles, one and several
# slabs with their scales, R not a multiple of 16.  Other modes (MN-major
# tiles, v a multiple of 8): mode 0 (the slab scales folded into X), ragged
# v tiles (a half-empty second box), ragged n_k, order 4.
TC_CASES = [((20480, 64), 1, 8), ((19500, 200), 1, 13), ((4, 5000, 1024), 2, 16), ((2, 9781, 8), 2, 33),
            ((19457, 520), 1, 64),
            ((300, 20480), 0, 16), ((40, 96, 520), 1, 8), ((160, 33, 64), 1, 21), ((2, 80, 130, 128), 2, 64),
            ((8, 64, 2432), 0, 24)]


@pytest.mark.parametrize("dims,k,R", TC_CASES,
                         ids=lambda c: "x".join(map(str, c)) if isinstance(c, tuple) else str(c))
def test_tmc_tensor_core_bf16(dims, k, R):
    A, Ao, scales = gu.inputs(dims, oracle.BF16, seed=5)
    X = mat(oracle.BF16, R, dims[k], synth.stream_x(k), seed=6)
    ref = oracle.tmc(Ao, k, X, scales=scales)
    launches0 = tg.kernel_launches()
    got = gpu_tmc(A, k, X, scales=scales, dims=dims)
    torch.cuda.synchronize()
    assert tg.kernel_launches() - launches0 == 2  # split of X + the tensor-core kernel
    assert gu.rel_l2(got, ref) <= 1e-5, (dims, R, gu.rel_l2(got, ref))
    lib = tg.load_library()
    import ctypes
    code = ctypes.c_int(0)
    assert lib.tvc_device_error(ctypes.byref(code), 1) == 0, code.value


def test_tmc_tensor_core_alpha_beta():
    dims, R = (20000, 128), 24
    A, Ao, scales = gu.inputs(dims, oracle.BF16, seed=7)
    X = mat(oracle.BF16, R, 128, synth.stream_x(1), seed=8)
    Y0 = synth.tensor("u32", 9, (20000, R)).astype(np.float32)
    ref = oracle.tmc(Ao, 1, X, scales=scales, Y=Y0.astype(np.float64), alpha=0.5, beta=-2.0)
    Yt = gu.to_dev(Y0)
    tg.tmc(gu.to_dev(A), 1, gu.to_dev(X), Y=Yt, scales=gu.to_dev(scales), shape=dims, alpha=0.5, beta=-2.0)
    torch.cuda.synchronize()
    assert gu.rel_l2(Yt.cpu().numpy(), ref) <= 1e-5


# FP32 storage: tf32 tensor-core MMAs on A, its low part A - trunc(A)
# written by converter warps, and the two parts of X; FP32 tolerance against
# the oracle.  Last mode (n_k a multiple of 4, K-major tiles) and the other
# modes (v a multiple of 4, MN-major tiles of four 32-wide boxes).
# FP32: rows of the last mode (TMA tiles, n_k % 4 == 0, R >= 8) as for BF16;
# other modes (R > 8, v >= 32 and v % 4 == 0, the slabs read by the converter
# warps): a part-filled last tile, ragged n_k, order 4.
TC_F32_CASES = [((20480, 64), 1, 8), ((19500, 200), 1, 13), ((4, 5000, 1024), 2, 16), ((2, 9781, 12), 2, 33),
                ((19457, 520), 1, 64),
                ((300, 20480), 0, 16), ((40, 96, 520), 1, 9), ((160, 33, 64), 1, 21), ((2, 80, 130, 128), 2, 64),
                ((8, 64, 2432), 0, 24), ((160, 37, 52), 1, 12), ((8, 200, 70, 34), 1, 40), ((97, 300, 132), 1, 17)]


@pytest.mark.parametrize("dims,k,R", TC_F32_CASES,
                         ids=lambda c: "x".join(map(str, c)) if isinstance(c, tuple) else str(c))
def test_tmc_tensor_core_f32(dims, k, R):
    A, Ao, _ = gu.inputs(dims, oracle.F32, seed=5)
    X = mat(oracle.F32, R, dims[k], synth.stream_x(k), seed=6)
    ref = oracle.tmc(Ao, k, X)
    launches0 = tg.kernel_launches()
    got = gpu_tmc(A, k, X, dims=dims)
    torch.cuda.synchronize()
    assert tg.kernel_launches() - launches0 == 2  # split of X + the tensor-core kernel
    code = ctypes.c_int(0)
    assert tg.load_library().tvc_device_error(ctypes.byref(code), 1) == 0, code.value
    assert code.value == 0, code.value  # no bounded wait ran out
    assert gu.rel_l2(got, ref) <= 1e-5, (dims, R, gu.rel_l2(got, ref))


def test_tmc_tensor_core_f32_alpha_beta():
    dims, R = (20000, 128), 24
    A, Ao, _ = gu.inputs(dims, oracle.F32, seed=7)
    X = mat(oracle.F32, R, 128, synth.stream_x(1), seed=8)
    Y0 = synth.tensor("u32", 9, (20000, R)).astype(np.float32)
    ref = oracle.tmc(Ao, 1, X, Y=Y0.astype(np.float64), alpha=0.5, beta=-2.0)
    Yt = gu.to_dev(Y0)
    tg.tmc(gu.to_dev(A), 1, gu.to_dev(X), Y=Yt, shape=dims, alpha=0.5, beta=-2.0)
    torch.cuda.synchronize()
    assert gu.rel_l2(Yt.cpu().numpy(), ref) <= 1e-5
