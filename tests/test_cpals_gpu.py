"""GPU parity of the CP-ALS building blocks (through the C ABI) against the
FP64 oracle: the Khatri-Rao product, and the MTTKRP for every mode and
storage type with either side of the mode contracted first, mode 0, the
last mode, leading modes of size one, order 1, and R across one and
several passes of the tensor-matrix contraction.

Tolerances (relative l2): FP64 and single-double 1e-12, FP32 and the narrow
types (against the oracle on the same codes) 1e-5."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

CODES = [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16]
SHAPES = [(7,), (5, 6), (3, 4, 5), (40, 3, 6), (6, 3, 40), (1, 1, 9, 4), (2, 3, 4, 3, 2), (9, 33, 130),
          (130, 33, 9), (50, 1000), (1000, 50), (4, 1, 7)]


@pytest.mark.parametrize("vt", [np.float64, np.float32], ids=["f64", "f32"])
def test_khatri_rao(vt):
    for rows in ((3,), (3, 5), (4, 1, 6), (2, 3, 2, 5)):
        for R in (1, 4, 9):
            mats = [synth.tensor("u64", 1, (n, R), 10 + m).astype(vt) for m, n in enumerate(rows)]
            got = tg.khatri_rao([gu.to_dev(U) for U in mats]).cpu().numpy()
            ref = oracle.khatri_rao(mats)
            tol = 1e-15 if vt == np.float64 else 1e-6
            assert got.shape == ref.shape
            assert gu.rel_l2(got, ref) <= tol, (rows, R)


def factors_for(dims, R, vt, seed=3):
    return [synth.tensor("u64", seed, (n, R), 20 + m).astype(vt) for m, n in enumerate(dims)]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_mttkrp_every_mode(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    vt = np.float64 if code == oracle.F64 else np.float32
    for k in range(len(dims)):
        for R in (1, 3, 8, 13):
            X = factors_for(dims, R, vt)
            ref = oracle.mttkrp(Ao, k, X, R=R, scales=scales)
            got = tg.mttkrp(gu.to_dev(A), k, [None if m == k else gu.to_dev(X[m]) for m in range(len(dims))], R=R,
                            scales=gu.to_dev(scales) if scales is not None else None, shape=dims).cpu().numpy()
            assert got.shape == ref.shape == (dims[k], R)
            assert gu.rel_l2(got, ref) <= gu.TOL[code], (dims, k, R)


@pytest.mark.parametrize("dims", [(3, 4, 5), (40, 3, 6), (6, 3, 40), (1, 1, 9, 4)], ids=lambda d: "x".join(map(str, d)))
def test_mttkrp_single_double(dims):
    A = synth.tensor("u32", 2, dims)
    for k in range(len(dims)):
        X = factors_for(dims, 5, np.float64)
        got = tg.mttkrp(gu.to_dev(A), k, [None if m == k else gu.to_dev(X[m]) for m in range(len(dims))],
                        shape=dims).cpu().numpy()
        assert got.dtype == np.float64
        assert gu.rel_l2(got, oracle.mttkrp(A, k, X)) <= 1e-12, (dims, k)


def test_mttkrp_one_column_is_hopms_all_but_one_contraction():
    """R = 1 gives z_k = A x_{m != k} x_m, the contraction of the power method."""
    dims = (6, 7, 8)
    A = synth.tensor("u64", 5, dims)
    xs = [synth.vector("u64", 6, 30 + m, n) for m, n in enumerate(dims)]
    for k in range(3):
        T = A
        for m in reversed(range(3)):
            if m != k:
                T = oracle.tvc(T, m, xs[m])
        got = tg.mttkrp(gu.to_dev(A), k, [gu.to_dev(x[:, None].copy()) for x in xs]).cpu().numpy()
        assert gu.rel_l2(got[:, 0], T) <= 1e-12, k


@pytest.mark.parametrize("case", [((4, 96, 96, 96), 0), ((4, 96, 96, 96), 1), ((2, 5, 128, 8192), 1)],
                         ids=["4x96^3-k0", "4x96^3-k1", "2x5x128x8192-k1"])
@pytest.mark.parametrize("code", [oracle.F64, oracle.F32, oracle.BF16], ids=["f64", "f32", "bf16"])
def test_mttkrp_long_trailing_block(case, code):
    """Trailing modes whose transposed Khatri-Rao rows exceed the L2-sized
    budget: the pass over A contracts only a suffix of them and the rest
    goes to the finishing contraction with the lower factors."""
    dims, k = case
    A, Ao, scales = gu.inputs(dims, code)
    vt = np.float64 if code == oracle.F64 else np.float32
    R = 8
    X = factors_for(dims, R, vt)
    ref = oracle.mttkrp(Ao, k, X, R=R, scales=scales)
    got = tg.mttkrp(gu.to_dev(A), k, [None if m == k else gu.to_dev(X[m]) for m in range(len(dims))],
                    scales=gu.to_dev(scales) if scales is not None else None, shape=dims).cpu().numpy()
    assert gu.rel_l2(got, ref) <= gu.TOL[code], (dims, k)


def test_mttkrp_bad_arguments():
    A = gu.to_dev(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        tg.mttkrp(A, 0, [None, gu.to_dev(np.zeros((3, 2)))])
    with pytest.raises(ValueError):
        tg.mttkrp(A, 2, [None, gu.to_dev(np.zeros((4, 2)))])
    lib = tg.load_library()
    dims = tg._dims_array((3, 4))
    import ctypes
    F = gu.to_dev(np.zeros((4, 2)))
    ptrs = (ctypes.c_void_p * 2)(0, F.data_ptr())
    M = gu.to_dev(np.zeros((3, 2)))
    # no workspace, and R < 1
    assert lib.mttkrp(tg._ptr(A), 2, dims, 0, ptrs, 2, tg._ptr(M), tg.F64, None, None, 0, None) != 0
    assert lib.mttkrp(tg._ptr(A), 2, dims, 0, ptrs, 0, tg._ptr(M), tg.F64, None, None, 0, None) != 0
