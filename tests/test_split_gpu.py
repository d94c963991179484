"""GPU parity of the 1D split over virtual ranks (Section 3.1: dTVC, Eq. 1
and Eq. 2; Algorithm 1: dHOPM_3) against the FP64 oracle on the unsplit
tensor, through the C ABI.

Tolerances as for the unsplit paths: TVC FP64 1e-12, FP32 and narrow
storage 1e-5 (relative l2); HOPM lambda history 1e-12 (FP64) / 1e-5, x_j
within 1e-10 / 2e-4.  Slab copies are bit-exact; one rank reproduces the
unsplit HOPM bit for bit.
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

CODES = [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16]
IDS = ["f64", "f32", "bf16", "e4m3", "f16"]


def _dev_codes(A):
    return gu.to_dev(A)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.int16, torch.uint8])
@pytest.mark.parametrize("dims", [(5, 7, 9), (3, 1, 4, 6), (17, 33), (2, 3, 4)])
def test_slab_copy_round_trip(dims, dtype):
    rng = np.random.default_rng(1)
    if dtype.is_floating_point:
        A = torch.from_numpy(rng.standard_normal(dims)).to(dtype)
    else:
        A = torch.from_numpy(rng.integers(0, 100, size=dims)).to(dtype)
    At = A.to(gu.DEV)
    for s in range(len(dims)):
        for p in (1, 2, 3):
            starts = tg.split_1d(dims[s], p)
            slabs = tg.split_tensor(At, s, starts)
            back = torch.zeros_like(At)
            for r, sl in enumerate(slabs):
                ref = A.narrow(s, starts[r], starts[r + 1] - starts[r])
                assert torch.equal(sl.cpu(), ref)
                tg.slab_insert(sl, back, s, starts[r], starts[r + 1])
            assert torch.equal(back.cpu(), A)


def test_slab_copy_misaligned_base():
    A = torch.arange(3 * 10 * 6 + 1, dtype=torch.float32, device=gu.DEV)[1:]  # 4-byte aligned only
    for s in range(3):
        sl = tg.slab_extract(A, s, 1, 3, shape=(3, 10, 6))
        ref = A.view(3, 10, 6).narrow(s, 1, 2)
        assert torch.equal(sl, ref.contiguous())


SPLIT_SHAPES = [(6, 5, 4), (7, 3, 5, 2), (13, 40), (2, 9, 3, 4, 2), (40, 64, 33)]


@pytest.mark.parametrize("dims", SPLIT_SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=IDS)
def test_dtvc_matches_unsplit_oracle(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    At = _dev_codes(A)
    st = gu.to_dev(scales) if scales is not None else None
    for s in range(len(dims)):
        for p in (1, 2, 3, 4):
            starts = tg.split_1d(dims[s], p)
            slabs = tg.split_tensor(At, s, starts, shape=dims)
            for k in range(len(dims)):
                x = gu.vec(code, dims[k], synth.stream_x(k))
                ref = oracle.tvc(Ao, k, x, scales=scales)
                got = tg.dtvc(slabs, starts, dims, s, k, gu.to_dev(x), scales=st)
                if k == s:  # Eq. 2: summed partials
                    assert gu.rel_l2(got.cpu().numpy(), ref) <= gu.TOL[code], (s, p, k)
                else:  # Eq. 1: disjoint output slabs along s (s - 1 past k)
                    so = s if s < k else s - 1
                    for r, yr in enumerate(got):
                        part = np.take(ref, np.arange(starts[r], starts[r + 1]), axis=so)
                        assert yr.shape == part.shape
                        assert gu.rel_l2(yr.cpu().numpy(), part) <= gu.TOL[code], (s, p, k, r)


@pytest.mark.parametrize("code", [oracle.F64, oracle.F32])
def test_dtvc_alpha_beta(code):
    dims = (5, 8, 6)
    A, Ao, _ = gu.inputs(dims, code)
    At = gu.to_dev(A)
    for s in range(3):
        starts = tg.split_1d(dims[s], 3)
        slabs = tg.split_tensor(At, s, starts)
        for k in range(3):
            x = gu.vec(code, dims[k], 1)
            out_dims = [n for i, n in enumerate(dims) if i != k]
            y0 = gu.vec(code, int(np.prod(out_dims)), 2).reshape(out_dims)
            ref = oracle.tvc(Ao, k, x, y=y0, alpha=0.5, beta=-2.0)
            if k == s:
                yt = gu.to_dev(y0)
                tg.dtvc(slabs, starts, dims, s, k, gu.to_dev(x), y=yt, alpha=0.5, beta=-2.0)
                assert gu.rel_l2(yt.cpu().numpy(), ref) <= gu.TOL[code]
            else:
                so = s if s < k else s - 1
                ys = [gu.to_dev(np.take(y0, np.arange(starts[r], starts[r + 1]), axis=so))
                      for r in range(len(starts) - 1)]
                tg.dtvc(slabs, starts, dims, s, k, gu.to_dev(x), y=ys, alpha=0.5, beta=-2.0)
                for r, yr in enumerate(ys):
                    part = np.take(ref, np.arange(starts[r], starts[r + 1]), axis=so)
                    assert gu.rel_l2(yr.cpu().numpy(), part) <= gu.TOL[code]


def test_dtvc_integer_inputs_bit_exact():
    rng = np.random.default_rng(3)
    dims = (6, 10, 7)
    A = rng.integers(-500, 500, size=dims).astype(np.float64)
    At = gu.to_dev(A)
    for s in range(3):
        starts = tg.split_1d(dims[s], 4)
        slabs = tg.split_tensor(At, s, starts)
        for k in range(3):
            x = rng.integers(-500, 500, size=dims[k]).astype(np.float64)
            ref = oracle.tvc(A, k, x)
            got = tg.dtvc(slabs, starts, dims, s, k, gu.to_dev(x))
            if k == s:
                assert np.array_equal(got.cpu().numpy(), ref)
            else:
                so = s if s < k else s - 1
                whole = np.concatenate([g.cpu().numpy() for g in got], axis=so)
                assert np.array_equal(whole, ref)


def _ones(dims, code):
    vt = torch.float64 if code == oracle.F64 else torch.float32
    return [torch.full((n,), 1.0 / math.sqrt(n), dtype=vt, device=gu.DEV) for n in dims]


HOPM_SHAPES = [(9, 7), (5, 6, 7), (4, 5, 3, 6), (3, 4, 2, 3, 5), (40, 33, 20)]


@pytest.mark.parametrize("dims", HOPM_SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=IDS)
def test_dhopm_matches_unsplit_oracle(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    iters = 6
    ref = oracle.hopm(Ao, [np.ones(n) / math.sqrt(n) for n in dims], iters, scales=scales)
    assert ref["status"] == 0
    At = _dev_codes(A)
    st = gu.to_dev(scales) if scales is not None else None
    tol = 1e-12 if code == oracle.F64 else 1e-5
    xtol = 1e-10 if code == oracle.F64 else 2e-4
    for s in range(len(dims)):
        for p in (2, 3):
            starts = tg.split_1d(dims[s], p)
            slabs = tg.split_tensor(At, s, starts, shape=dims)
            r = tg.dhopm(slabs, starts, dims, s, _ones(dims, code), iters, scales=st)
            torch.cuda.synchronize()
            assert int(r.status.item()) == 0
            assert int(r.sweeps.item()) == iters
            np.testing.assert_allclose(r.lam_hist.cpu().numpy()[:iters], ref["lam_hist"], rtol=tol)
            for xg, xr in zip(r.x, ref["x"]):
                assert np.max(np.abs(xg.cpu().numpy().astype(np.float64) - xr)) <= xtol, (s, p)


@pytest.mark.parametrize("code", [oracle.F64, oracle.F32])
def test_dhopm_one_rank_equals_hopm_bitwise(code):
    dims = (12, 10, 8, 6)
    A, _, _ = gu.inputs(dims, code)
    At = gu.to_dev(A)
    a = tg.hopm(At, _ones(dims, code), 5)
    for s in range(4):
        b = tg.dhopm([At], [0, dims[s]], dims, s, _ones(dims, code), 5)
        torch.cuda.synchronize()
        assert torch.equal(a.lam_hist, b.lam_hist)
        for xa, xb in zip(a.x, b.x):
            assert torch.equal(xa, xb)


def test_dhopm_stopping_rule_and_zero_status():
    dims = (8, 9, 10)
    A = synth.tensor("u64", 5, dims)
    ref = oracle.hopm(A, [np.ones(n) / math.sqrt(n) for n in dims], 50, 1e-9)
    At = gu.to_dev(A)
    starts = tg.split_1d(dims[1], 3)
    slabs = tg.split_tensor(At, 1, starts)
    r = tg.dhopm(slabs, starts, dims, 1, _ones(dims, oracle.F64), 50, 1e-9)
    torch.cuda.synchronize()
    assert int(r.sweeps.item()) == ref["sweeps"]
    assert abs(r.lam.item() - ref["lam"]) <= 1e-12 * ref["lam"]
    # a zero tensor: zero norm on the first update, status set, run stopped
    Z = torch.zeros(dims, dtype=torch.float64, device=gu.DEV)
    zs = tg.split_tensor(Z, 0, tg.split_1d(8, 2))
    r = tg.dhopm(zs, tg.split_1d(8, 2), dims, 0, _ones(dims, oracle.F64), 5)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 5  # TVC_ERR_ZERO_NORM


def test_split_bad_arguments_raise():
    At = torch.zeros((4, 6), dtype=torch.float64, device=gu.DEV)
    x = torch.zeros(6, dtype=torch.float64, device=gu.DEV)
    slabs = tg.split_tensor(At, 0, [0, 2, 4])
    with pytest.raises(tg.TVCError):  # starts do not end at n_s
        tg.dtvc(slabs, [0, 2, 3], (4, 6), 0, 1, x)
    with pytest.raises(tg.TVCError):  # s out of range
        tg.dtvc(slabs, [0, 2, 4], (4, 6), 2, 1, x)
    with pytest.raises(ValueError):
        tg.split_1d(0, 2)


def test_split_single_double():
    dims = (7, 3, 5, 2)
    A = synth.tensor("u32", 1, dims)
    At = gu.to_dev(A)
    for s in range(len(dims)):
        starts = tg.split_1d(dims[s], 3)
        slabs = tg.split_tensor(At, s, starts)
        for k in range(len(dims)):
            x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
            ref = oracle.tvc(A, k, x)
            got = tg.dtvc(slabs, starts, dims, s, k, gu.to_dev(x))
            if k == s:
                assert gu.rel_l2(got.cpu().numpy(), ref) <= 1e-12
            else:
                so = s if s < k else s - 1
                assert gu.rel_l2(np.concatenate([g.cpu().numpy() for g in got], axis=so), ref) <= 1e-12
        r = tg.dhopm(slabs, starts, dims, s, _ones(dims, oracle.F64), 5)
        ref = oracle.hopm(A, [np.ones(n) / math.sqrt(n) for n in dims], 5)
        torch.cuda.synchronize()
        np.testing.assert_allclose(r.lam_hist.cpu().numpy()[:5], ref["lam_hist"], rtol=1e-12)
