"""GPU parity of the TVC adjoints (through the C ABI and the autograd
wrapper) against the oracle's gradients, central finite differences and
the adjoint identity <gy, A x_k x> = <gx, x> = <gA, A>."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

SHAPES = [(7,), (5, 3), (4, 1), (3, 1, 5), (6, 5, 4, 3), (3, 50, 64), (5, 1000), (4, 100, 7), (300, 40),
          (50, 8, 8), (2000, 64), (9, 33, 130), (2, 3, 2, 3, 2, 3, 2), (257, 1, 3)]
CODES = [oracle.F64, oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("code", CODES, ids=["f64", "f32", "bf16", "e4m3", "f16"])
def test_backward_matches_oracle(dims, code):
    A, Ao, scales = gu.inputs(dims, code)
    for k in range(len(dims)):
        x = gu.vec(code, dims[k], synth.stream_x(k))
        gyshape = [n for i, n in enumerate(dims) if i != k]
        gy = gu.vec(code, int(np.prod(gyshape, dtype=np.int64)), 40 + k).reshape(gyshape)
        gx, gA = tg.tvc_backward(gu.to_dev(A), k, gu.to_dev(x), gu.to_dev(gy), shape=dims,
                                 scales=gu.to_dev(scales) if scales is not None else None,
                                 need_A=code in (oracle.F64, oracle.F32))
        ref_gx = oracle.tvc_grad_x(Ao, k, gy, scales=scales)
        assert gu.rel_l2(gx.cpu().numpy(), ref_gx) <= gu.TOL[code], (dims, k)
        if gA is not None:
            ref_gA = oracle.tvc_grad_A(dims, k, x, gy)
            assert gu.rel_l2(gA.cpu().numpy(), ref_gA) <= gu.TOL[code], (dims, k)


def test_gradA_accumulate():
    dims = (4, 6, 40)
    A = synth.tensor("u64", 1, dims)
    for k in range(3):
        x = synth.vector("u64", 2, 1, dims[k])
        gy = synth.vector("u64", 3, 2, A.size // dims[k])
        g0 = synth.tensor("u64", 4, dims)
        gAt = gu.to_dev(g0)
        tg.tvc_backward(gu.to_dev(A), k, gu.to_dev(x), gu.to_dev(gy), need_x=False, gA=gAt, beta_A=0.5)
        ref = oracle.tvc_grad_A(dims, k, x, gy) + 0.5 * g0
        assert gu.rel_l2(gAt.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("dims", [(4, 5, 3), (6, 7), (2, 3, 2, 3), (5, 40, 33)])
def test_autograd_finite_differences_and_adjoint_identity(dims):
    A = gu.to_dev(synth.tensor("u64", 5, dims)).requires_grad_(True)
    for k in range(len(dims)):
        x = gu.to_dev(synth.vector("u64", 6, 1, dims[k])).requires_grad_(True)
        gyshape = [n for i, n in enumerate(dims) if i != k]
        gy = gu.to_dev(synth.tensor("u64", 7, gyshape))
        y = tg.tvc_autograd(A, x, k)
        L = (y * gy).sum()
        gA, gx = torch.autograd.grad(L, (A, x))
        # adjoint identity
        lhs = float(L)
        assert abs(lhs - float(torch.dot(gx, x))) <= 1e-12 * max(1.0, abs(lhs))
        assert abs(lhs - float((gA * A).sum())) <= 1e-12 * max(1.0, abs(lhs))
        # central finite differences through the GPU forward
        h = 1e-6
        with torch.no_grad():
            for j in range(min(dims[k], 5)):
                e = torch.zeros_like(x)
                e[j] = h
                fd = (float((tg.tvc(A, k, x + e) * gy).sum()) - float((tg.tvc(A, k, x - e) * gy).sum())) / (2 * h)
                assert abs(fd - float(gx[j])) <= 1e-7 * max(1.0, abs(fd))
            flat = A.detach().reshape(-1)
            for f in (0, flat.numel() // 3, flat.numel() - 1):
                Ap = flat.clone(); Ap[f] += h
                Am = flat.clone(); Am[f] -= h
                fd = (float((tg.tvc(Ap.reshape(dims), k, x) * gy).sum()) -
                      float((tg.tvc(Am.reshape(dims), k, x) * gy).sum())) / (2 * h)
                assert abs(fd - float(gA.reshape(-1)[f])) <= 1e-7


def test_backward_deterministic():
    dims = (30, 500, 40)
    A = gu.to_dev(synth.tensor("u64", 8, dims))
    x = gu.to_dev(synth.vector("u64", 8, 1, 500))
    gy = gu.to_dev(synth.vector("u64", 8, 2, 30 * 40))
    a, _ = tg.tvc_backward(A, 1, x, gy, need_A=False)
    b, _ = tg.tvc_backward(A, 1, x, gy, need_A=False)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: "x".join(map(str, d)))
def test_backward_single_double(dims):
    """binary32 storage, FP64 vectors and arithmetic (single-double)."""
    A = synth.tensor("u32", 2, dims)
    for k in range(len(dims)):
        x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
        gyshape = [n for i, n in enumerate(dims) if i != k]
        gy = synth.vector("u64", 3, 40 + k, int(np.prod(gyshape, dtype=np.int64))).reshape(gyshape)
        gx, gA = tg.tvc_backward(gu.to_dev(A), k, gu.to_dev(x), gu.to_dev(gy), shape=dims)
        assert gx.dtype == torch.float64 and gA.dtype == torch.float64
        assert gu.rel_l2(gx.cpu().numpy(), oracle.tvc_grad_x(A, k, gy)) <= 1e-12, (dims, k)
        assert gu.rel_l2(gA.cpu().numpy(), oracle.tvc_grad_A(dims, k, x, gy)) <= 1e-12, (dims, k)
