"""GPU parity of the TVC kernels (through the C ABI) against the FP64 oracle.

Tolerances (relative l2 over the output): FP64 1e-12, FP32 1e-5; narrow
storage: the kernel against the oracle on the same stored codes 1e-5 (FP32
accumulation), and the stored tensor against its FP32 source (storage error)
2e-2 for BF16.  Integer-valued FP64 inputs must match bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

# Shapes chosen to reach every kernel of the contraction: COLS (v >= 32),
# ROWS (v == 1, long rows), SLAB (1 < v < 32, large slabs), TILE (small
# slabs), with split-K (few outputs, long n_k), ragged sizes and tails.
SHAPES = [
    (7,), (100003,), (5, 3), (1, 4), (4, 1), (3, 1, 5), (2, 3, 4), (6, 5, 4, 3), (2, 1, 3, 1, 2),
    (3, 50, 64), (5, 1000), (3, 4099), (4, 100, 7), (300, 40), (50, 8, 8), (2000, 64), (13, 17, 19, 3),
    (9, 33, 130), (2, 3, 2, 3, 2, 3, 2), (1, 1, 1), (257, 1, 3),
    # long rows with 16-byte pieces (several rows per warp): ragged row
    # counts, a single row, split-K, and mode 0 of an order-1 tensor
    (7, 3072), (19, 2, 1040), (1, 4096), (2048,), (3, 65536), (1001, 1536),
    # large slabs with 1 < v < 32 (staged 16-byte tiles for the narrow
    # types, 4, 2 or 1 columns per thread): v = 16, 12, 7, 31 and 2, ragged
    # n_k, split n_k
    (3, 600, 16), (2, 300, 12), (5, 3000, 7), (3, 700, 31), (6, 4099, 2),
    # short rows of 8 .. 27 elements (FP64: the copy-engine tile kernel,
    # padded 2-D boxes for lengths 0 mod 4; single-double: shared-memory
    # tiles or the grouped-row kernel), ragged last tiles, one partial tile
    (1001, 10), (777, 19), (513, 22), (257, 27), (300, 12), (100, 9), (600, 16), (600, 8),
    # large slabs whose rows are whole 16-byte pieces (the copy-engine slab
    # kernel for FP32 and the narrow types): ragged tiles, one slab split
    # over its rows, mode 0 of a matrix (slab scales folded into x)
    (7, 1000, 8), (1, 4096, 16), (33, 300, 16), (4096, 16), (5, 4099, 4),
    # columns with short contractions (n_k <= 32, v >= 32): odd and even v,
    # ragged thread tails, n_k of 1 .. 32
    (13, 13, 13, 13), (10, 10, 10, 10), (3, 32, 67), (5, 1, 99), (31, 97), (2, 7, 1000),
]
CODES = [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_tvc_every_mode(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    for k in range(len(dims)):
        x = gu.vec(code, dims[k], synth.stream_x(k))
        ref = oracle.tvc(Ao, k, x, scales=scales)
        got = gu.gpu_tvc(tg, A, k, x, scales)
        assert got.shape == ref.shape
        err = gu.rel_l2(got, ref)
        assert err <= gu.TOL[code], (dims, k, err)


# FP64 small slabs and short rows through the copy-engine tile kernel: rows
# of odd length or of length 2 mod 4 for every lanes-per-output count
# (G = 1 .. 32), rows of length 0 mod 4 (padded 2-D boxes, zero rows past
# the tensor), slabs with 1 < v < 32, tensors of fewer slabs than one tile,
# ragged last tiles and odd element counts (the last element copied by hand)
F64_TILE_SHAPES = [(1001, 3), (4001, 2), (2003, 31), (999, 63), (2001, 175), (301, 333), (257, 767), (5, 10),
                   (3, 7), (1, 9), (1003, 6), (777, 3, 5), (2001, 9, 2), (101, 31, 31), (37, 40, 20),
                   (1999, 4, 3), (3, 5, 17), (1001, 8), (257, 16), (999, 24), (1001, 4), (77, 128), (3, 8),
                   (5, 20), (2049, 40), (301, 2, 12),
                   # FP64 rows of odd length beyond the tile kernel: 16-byte
                   # pairs from each row's first 16-byte boundary (split n_k too)
                   (7, 1001), (4, 4097), (3, 100001), (9, 2049), (2, 30623)]


@pytest.mark.parametrize("dims", F64_TILE_SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_fp64_tile_kernel_shapes(dims):
    import ctypes
    lib = tg.load_library()
    code = ctypes.c_int(-1)
    lib.tvc_device_error(ctypes.byref(code), 1)
    A = synth.tensor("u64", 9, dims)
    mode = len(dims) - 1 if len(dims) == 2 else 1
    for k in sorted({mode, 0, len(dims) - 1}):
        x = synth.vector("u64", 9, synth.stream_x(k), dims[k])
        got = gu.gpu_tvc(tg, A, k, x)
        assert gu.rel_l2(got, oracle.tvc(A, k, x)) <= 1e-12, (dims, k)
    rng = np.random.default_rng(sum(dims))
    Ai = rng.integers(-1000, 1000, size=dims).astype(np.float64)
    xi = rng.integers(-1000, 1000, size=dims[mode]).astype(np.float64)
    assert np.array_equal(gu.gpu_tvc(tg, Ai, mode, xi), oracle.tvc(Ai, mode, xi)), dims
    torch.cuda.synchronize()
    assert lib.tvc_device_error(ctypes.byref(code), 0) == 0 and code.value == 0


@pytest.mark.parametrize("dims", [(3, 50, 64), (5, 1000), (4, 100, 7), (300, 40)])
def test_narrow_storage_error_vs_source(dims):
    src = synth.tensor("lognormal", 0, dims).astype(np.float32)
    for code, bound in ((oracle.BF16, 2e-2), (oracle.E4M3, None), (oracle.F16, 2e-3)):
        codes, scales = oracle.quantise(src, code)
        for k in range(len(dims)):
            x = gu.vec(code, dims[k], synth.stream_x(k))
            got = gu.gpu_tvc(tg, codes, k, x, scales)
            err_src = gu.rel_l2(got, oracle.tvc(src, k, x))
            print(f"storage error {['f64','f32','bf16','e4m3','f16'][code]} {dims} mode {k}: {err_src:.3e}")
            if bound is not None:
                assert err_src <= bound
            else:
                assert err_src <= 0.1


@pytest.mark.parametrize("dims", [(6, 70, 33), (5, 1000), (4, 100, 7), (300, 40), (3, 50, 64), (2000, 64)])
def test_integer_inputs_bit_exact_f64(dims):
    rng = np.random.default_rng(11)
    A = rng.integers(-1000, 1000, size=dims).astype(np.float64)
    for k in range(len(dims)):
        x = rng.integers(-1000, 1000, size=dims[k]).astype(np.float64)
        ref = oracle.tvc(A, k, x)
        got = gu.gpu_tvc(tg, A, k, x)
        assert np.array_equal(got, ref), (dims, k)


# shapes reaching the column, slab (1 < v < 32, large slabs), small-slab
# (tile), odd short-row (8-byte loads) and even short-row kernels
WINDOW_SHAPES = [(40, 37, 66), (500, 19, 19), (40, 600, 12), (3000, 13), (2001, 175), (300, 40), (1001, 10), (777, 22),
                 (13, 13, 13, 13), (10, 10, 10, 10)]


@pytest.mark.parametrize("dims", WINDOW_SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_fp64_values_outside_the_emulation_window(dims):
    A = synth.tensor("u64", 4, dims)
    flat = A.ravel()
    rng = np.random.default_rng(5)
    pos = rng.choice(flat.size, size=600, replace=False)
    flat[pos[:100]] = 0.0
    flat[pos[100:200]] *= 1e300
    flat[pos[200:300]] *= 1e-300
    flat[pos[300:400]] = 5e-324  # subnormal
    flat[pos[400:500]] *= 2.0 ** 70
    flat[pos[500:]] *= 2.0 ** -70
    for k in range(len(dims)):
        x = synth.vector("u64", 1, 1 + k, dims[k])
        x[::5] *= 1e-20
        x[1::7] = 0.0
        ref = oracle.tvc(A, k, x)
        got = gu.gpu_tvc(tg, A, k, x)
        assert gu.rel_l2(got, ref) <= 1e-12, (dims, k)
        # and with x inside the window (only A's elements fall outside)
        x = synth.vector("u64", 1, 1 + k, dims[k])
        assert gu.rel_l2(gu.gpu_tvc(tg, A, k, x), oracle.tvc(A, k, x)) <= 1e-12, (dims, k)


@pytest.mark.parametrize("code", [oracle.F64, oracle.F32])
def test_alpha_beta(code):
    dims = (4, 33, 40)
    A, Ao, _ = gu.inputs(dims, code)
    for k in range(3):
        x = gu.vec(code, dims[k], 1)
        y0 = gu.vec(code, A.size // dims[k], 2).reshape([n for i, n in enumerate(dims) if i != k])
        ref = oracle.tvc(Ao, k, x, y=y0, alpha=0.5, beta=-2.0)
        yt = gu.to_dev(y0)
        tg.tvc(gu.to_dev(A), k, gu.to_dev(x), y=yt, alpha=0.5, beta=-2.0)
        assert gu.rel_l2(yt.cpu().numpy(), ref) <= gu.TOL[code]
        # beta == 0: y is not read
        yn = torch.full_like(yt, float("nan"))
        tg.tvc(gu.to_dev(A), k, gu.to_dev(x), y=yn, alpha=2.0, beta=0.0)
        assert gu.rel_l2(yn.cpu().numpy(), 2.0 * oracle.tvc(Ao, k, x)) <= gu.TOL[code]


@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_misaligned_base(code):
    dims = (6, 40, 48)
    A, Ao, scales = gu.inputs(dims, code)
    buf = torch.zeros(A.size + 1, dtype=gu.to_dev(A).dtype, device=gu.DEV)
    buf[1:] = gu.to_dev(A.ravel())
    At = buf[1:]
    for k in range(3):
        x = gu.vec(code, dims[k], synth.stream_x(k))
        st = gu.to_dev(scales) if scales is not None else None
        got = tg.tvc(At, k, gu.to_dev(x), scales=st, shape=dims).cpu().numpy()
        assert gu.rel_l2(got, oracle.tvc(Ao, k, x, scales=scales)) <= gu.TOL[code]


@pytest.mark.parametrize("dims,mode", [((20000, 64), 0), ((3, 300000), 1), ((1000003,), 0), ((2, 5000, 9), 1)])
def test_split_k_deterministic(dims, mode):
    A = synth.tensor("u64", 2, dims)
    x = synth.vector("u64", 3, 1, dims[mode])
    a = gu.gpu_tvc(tg, A, mode, x)
    b = gu.gpu_tvc(tg, A, mode, x)
    assert np.array_equal(a, b)
    assert gu.rel_l2(a, oracle.tvc(A, mode, x)) <= 1e-12


def test_empty_like_degenerate_sizes():
    # all-ones dims: a single element; order 1: a dot product
    for dims in [(1,), (1, 1), (1, 1, 1, 1)]:
        A = np.full(dims, 3.0)
        for k in range(len(dims)):
            got = gu.gpu_tvc(tg, A, k, np.array([2.0]))
            assert np.all(got == 6.0)


@pytest.mark.parametrize("dims", [(64, 2048), (8, 33, 512), (300, 4, 96)], ids=lambda d: "x".join(map(str, d)))
def test_e4m3_columns_with_large_and_nonfinite_x(dims):
    """E4M3 columns with x entries far from unit size (up to 2.5e6) give the
    oracle's values, and an infinite entry of x gives non-finite outputs
    exactly where the oracle's are."""
    src = synth.tensor("lognormal", 3, dims).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.E4M3)
    for k in range(len(dims)):
        x = gu.vec(oracle.E4M3, dims[k], synth.stream_x(k))
        x[::7] *= 300.0
        x[1] = -2.5e6
        x[2] = 255.99
        ref = oracle.tvc(codes, k, x, scales=scales)
        got = gu.gpu_tvc(tg, codes, k, x, scales)
        assert gu.rel_l2(got, ref) <= 1e-5, (dims, k)
        x[3] = np.inf
        got = gu.gpu_tvc(tg, codes, k, x, scales)
        ref = oracle.tvc(codes, k, x, scales=scales)
        assert np.array_equal(np.isfinite(got), np.isfinite(ref)), (dims, k)


@pytest.mark.parametrize("dims", [(3, 600, 16), (7, 1000, 16)], ids=lambda d: "x".join(map(str, d)))
def test_e4m3_nan_codes_in_slabs(dims):
    """E4M3 slabs (decoded with integer operations): a NaN code (S.1111.111)
    makes exactly the outputs it feeds NaN, as in the oracle's decode."""
    src = synth.tensor("lognormal", 5, dims).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.E4M3)
    flat = codes.reshape(-1)
    flat[[5, 16 * 37 + 3, 16 * 600 + 15]] = [0x7F, 0xFF, 0x7F]
    x = gu.vec(oracle.E4M3, dims[1], synth.stream_x(1))
    ref = oracle.tvc(codes, 1, x, scales=scales)
    got = gu.gpu_tvc(tg, codes, 1, x, scales)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = ~np.isnan(ref)
    assert gu.rel_l2(got[fin], ref[fin]) <= 1e-5


def test_bad_arguments_raise():
    A = gu.to_dev(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        tg.tvc(A, 2, gu.to_dev(np.zeros(4)))
    with pytest.raises(ValueError):
        tg.tvc(A, 0, gu.to_dev(np.zeros(4)))
    with pytest.raises(ValueError):
        tg.tvc(A, 1, gu.to_dev(np.zeros(4, dtype=np.float32)))


def test_config_128cube_fp64_all_modes():
    """Plain-method FP64 workload: 128^3, uniform[-1,1], seed 0, every mode."""
    dims = (128, 128, 128)
    A = synth.tensor("u64", 0, dims)
    At = gu.to_dev(A)
    for k in range(3):
        x = synth.vector("u64", 0, synth.stream_x(k), 128)
        ref = oracle.tvc(A, k, x)
        got = tg.tvc(At, k, gu.to_dev(x)).cpu().numpy()
        assert gu.rel_l2(got, ref) <= 1e-12


def test_device_generator_matches_host():
    import synth.device as sd
    for kind, dt in (("u64", torch.float64), ("u32", torch.float32), ("gauss", torch.float64),
                     ("lognormal", torch.float32)):
        t = torch.empty(5000, dtype=dt, device=gu.DEV)
        sd.fill(t, kind, 7, 3, offset=123456789)
        idx = np.arange(123456789, 123456789 + 5000, dtype=np.uint64)
        host = {"u64": synth.uniform_f64, "u32": synth.uniform_f32, "gauss": synth.gaussian_f64,
                "lognormal": synth.lognormal_mix_f64}[kind](7, 3, idx)
        assert np.array_equal(t.cpu().numpy(), host.astype(t.cpu().numpy().dtype)), kind
    dims = (5, 6, 7)
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    t = torch.empty(210, dtype=torch.float32, device=gu.DEV)
    sd.fill(t, "planted", 0, 0, dims=dims, us=us)
    assert np.array_equal(t.cpu().numpy(), synth.tensor("planted", 0, dims, us=us).astype(np.float32).ravel())


# Full-size bandwidth-sweep tensors: filled on the device from the same
# counter-based definition the host uses; outputs checked at sampled indices
# against the oracle computed from host-generated elements.
FULL = [(1024, 1024, 1024), (128, 128, 128, 128), (40, 40, 40, 40, 40, 40), (65536, 16384)]


@pytest.mark.slow
@pytest.mark.parametrize("dims", FULL, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", [oracle.F64, oracle.F32], ids=["f64", "f32"])
def test_full_size_sweep_sampled(dims, code):
    import synth.device as sd
    kind = "u64" if code == oracle.F64 else "u32"
    dt = torch.float64 if code == oracle.F64 else torch.float32
    N = int(np.prod(dims, dtype=np.int64))
    At = torch.empty(N, dtype=dt, device=gu.DEV)
    sd.fill(At, kind, 0, synth.STREAM_A)
    rng = np.random.default_rng(0)
    for k in range(len(dims)):
        x = gu.vec(code, dims[k], synth.stream_x(k), seed=1)
        y = tg.tvc(At, k, gu.to_dev(x), shape=dims)
        yf = y.reshape(-1)
        picks, u, v = gu.sample_outputs(dims, k, 48, rng)
        got = yf[torch.from_numpy(picks).to(gu.DEV)].cpu().numpy()
        ref, mag = gu.oracle_at(kind, 0, dims, k, x, picks, v, exact=code == oracle.F64)
        assert gu.rel_l2(got, ref) <= gu.TOL[code], (dims, k)
        if code == oracle.F64:  # the FP64 error model, against the exactly rounded sums
            assert np.all(np.abs(got - ref) <= gu.f64_model_bound(mag, dims[k]) + 2.0 ** -52 * np.abs(ref)), (dims, k)
        else:
            assert np.all(np.abs(got - ref) <= 50 * gu.TOL[code] * mag), (dims, k)
        assert bool(torch.isfinite(y).all())
        del y
    del At
    torch.cuda.empty_cache()


def test_staged_kernel_waits_never_time_out():
    """The copy-engine kernels (staged rows, FP64 tiles, slab tiles) bound
    every wait and record a timeout in a sticky device word; after runs over
    many tiles the word must be 0."""
    import ctypes
    lib = tg.load_library()
    code = ctypes.c_int(-1)
    lib.tvc_device_error(ctypes.byref(code), 1)  # clear
    for dims, dt in (((200000, 40), "u32"), ((4096, 128), "u32"), ((30001, 8), "u32"), ((64, 4096, 8), "u32"),
                     ((999, 63), "u64"), ((3000, 8), "u64")):
        A = synth.tensor(dt, 3, dims)
        x = synth.vector(dt, 4, 2, dims[1])
        got = gu.gpu_tvc(tg, A, 1, x)
        assert gu.rel_l2(got, oracle.tvc(A, 1, x)) <= 1e-5
    torch.cuda.synchronize()
    assert lib.tvc_device_error(ctypes.byref(code), 0) == 0 and code.value == 0


# ----------------------------------------------------- single-double (F32D)
# binary32 storage with FP64 vectors and FP64 arithmetic (Section 5.5): the
# oracle's FP32 path computes exactly that (elements promoted to FP64), so
# the FP64 tolerance applies.

@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_single_double_every_mode(dims):
    A = synth.tensor("u32", 0, dims)
    for k in range(len(dims)):
        x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
        got = gu.gpu_tvc(tg, A, k, x)
        assert got.dtype == np.float64
        assert gu.rel_l2(got, oracle.tvc(A, k, x)) <= 1e-12, (dims, k)


@pytest.mark.parametrize("dims", WINDOW_SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_single_double_outside_the_window(dims):
    A = synth.tensor("u32", 4, dims)
    flat = A.ravel()
    rng = np.random.default_rng(6)
    pos = rng.choice(flat.size, size=500, replace=False)
    flat[pos[:100]] = 0.0
    flat[pos[100:200]] = np.float32(1e38)
    flat[pos[200:300]] = np.float32(1e-40)  # subnormal
    flat[pos[300:400]] *= np.float32(2.0 ** 70)
    flat[pos[400:]] *= np.float32(2.0 ** -70)
    for k in range(len(dims)):
        x = synth.vector("u64", 1, 1 + k, dims[k])
        x[::5] *= 1e-20
        x[1::7] = 0.0
        assert gu.rel_l2(gu.gpu_tvc(tg, A, k, x), oracle.tvc(A, k, x)) <= 1e-12, (dims, k)


@pytest.mark.parametrize("dims", [(6, 70, 33), (5, 1000), (4, 100, 7), (3000, 13), (500, 19, 19)])
def test_single_double_integer_inputs_bit_exact(dims):
    rng = np.random.default_rng(12)
    A = rng.integers(-1000, 1000, size=dims).astype(np.float32)
    for k in range(len(dims)):
        x = rng.integers(-1000, 1000, size=dims[k]).astype(np.float64)
        assert np.array_equal(gu.gpu_tvc(tg, A, k, x), oracle.tvc(A, k, x)), (dims, k)


# --------------------------------------------------- FP64 error model

def cancelling(dims, mode, seed, kappa=1e6, lanes=1):
    """Uniform A and x (or an R x n_k matrix X when lanes = R > 1) with the
    last `lanes` slices of mode `mode` solved for so that every output (of
    every row of X) is about sum|a x| / kappa: sums that cancel heavily."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, dims)
    nk = dims[mode]
    X = rng.uniform(-1, 1, (lanes, nk))
    X[:, nk - lanes:] += 2.0 * np.eye(lanes)  # keep the solved system well conditioned
    u = int(np.prod(dims[:mode]))
    Ar = A.reshape(u, nk, -1)
    keep = nk - lanes
    part = np.einsum("ijl,rj->ilr", Ar[:, :keep, :], X[:, :keep])
    mag = np.einsum("ijl,rj->ilr", np.abs(Ar[:, :keep, :]), np.abs(X[:, :keep]))
    rhs = -(part - mag / kappa * rng.uniform(-1, 1, part.shape))
    sol = np.linalg.solve(X[:, keep:], rhs[..., None])[..., 0]  # (u, v, lanes)
    Ar[:, keep:, :] = np.transpose(sol, (0, 2, 1))
    return A, (X[0] if lanes == 1 else X)


# one shape per FP64 kernel (mode in brackets): columns (v >= 32, short and
# long n_k) and their split n_k, long rows and their split, odd long rows
# (16-byte pairs from each row's boundary, L1-sized segments), short rows
# and small slabs through the copy-engine tile kernel (G = 1 .. 16, padded
# rows of 8 and 128), large slabs with 1 < v < 32, unaligned tensors (the
# f64_unaligned store: the kernels that need no 16-byte alignment)
CANCEL_CASES = [((13, 13, 13, 13), 1), ((10, 10, 10, 10), 0), ((40, 37, 66), 1), ((3, 2000, 64), 1), ((300, 4096), 1), ((3, 300000), 1), ((3000, 40), 1),
                ((3000, 13), 1), ((2001, 175), 1), ((40, 600, 12), 1), ((500, 19, 19), 1), ((5, 3000, 7), 1),
                ((9, 33, 130), 0), ((6, 5, 4, 3), 2), ((999, 63), 1), ((101, 31, 31), 1), ((301, 333), 1),
                ((2049, 8), 1), ((301, 128), 1), ((7, 4097), 1), ((3, 100001), 1)]


@pytest.mark.parametrize("dims,mode", CANCEL_CASES, ids=lambda c: "x".join(map(str, c)) if isinstance(c, tuple) else str(c))
@pytest.mark.parametrize("store", ["f64", "f64_unaligned", "f32d"])
def test_fp64_error_model_on_cancelling_sums(dims, mode, store):
    """|y - y_exact| <= F64_MODEL_C 2^-46 sum|a x| (+ the FP64 block sum) on
    sums that cancel to about 1e-6 of sum|a x|, against the compensated
    oracle contraction; FP64 storage (16-byte aligned, and 8 bytes past
    that), and binary32 storage with FP64 arithmetic (single-double)."""
    A, x = cancelling(dims, mode, seed=sum(dims) + mode)
    if store == "f32d":
        A = A.astype(np.float32)
    ref = oracle.tvc_exact(A, mode, x)
    mag = oracle.tvc(np.abs(A.astype(np.float64)), mode, np.abs(x))
    if store == "f64_unaligned":
        buf = torch.empty(A.size + 1, dtype=torch.float64, device=gu.DEV)
        At = buf[1:]
        At.copy_(torch.from_numpy(A.ravel()))
    else:
        At = gu.to_dev(A.ravel())
    got = tg.tvc(At, mode, gu.to_dev(x), shape=dims).cpu().numpy()
    err = np.abs(got - ref)
    bound = gu.f64_model_bound(mag, dims[mode]) + 2.0 ** -52 * np.abs(ref)
    print(f"{store} {dims} mode {mode}: max |err| / (2^-46 sum|ax|) = {np.max(err / (2.0 ** -46 * mag)):.3f}")
    assert np.all(err <= bound), np.max(err / (2.0 ** -46 * mag))


@pytest.mark.parametrize("dims,mode", [((40, 37, 66), 1), ((3000, 40), 1), ((500, 19, 19), 1), ((3, 5000, 9), 1)],
                         ids=lambda c: "x".join(map(str, c)) if isinstance(c, tuple) else str(c))
def test_fp64_tmc_error_model_on_cancelling_sums(dims, mode):
    """The FP64 tensor-matrix contraction (float-float pieces, R = 2 rows of
    X, both cancelling) under the same error model, row by row against the
    compensated oracle contraction."""
    A, X = cancelling(dims, mode, seed=7 + mode, lanes=2)
    Y = tg.tmc(gu.to_dev(A), mode, gu.to_dev(X)).cpu().numpy()
    u = int(np.prod(dims[:mode]))
    Yr = Y.reshape(u, 2, -1)
    for r in range(2):
        ref = oracle.tvc_exact(A, mode, X[r]).reshape(u, -1)
        mag = oracle.tvc(np.abs(A), mode, np.abs(X[r])).reshape(u, -1)
        err = np.abs(Yr[:, r, :] - ref)
        assert np.all(err <= gu.f64_model_bound(mag, dims[mode]) + 2.0 ** -52 * np.abs(ref)), \
            np.max(err / (2.0 ** -46 * mag))
