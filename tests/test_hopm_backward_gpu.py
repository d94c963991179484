"""GPU HOPM backward (recomputation) against central finite differences of
the FP64 oracle's power method (FP64, FP32 and narrow storage), and the
envelope theorem at a fixed point: d lambda / dA = x_0 (x) ... (x) x_{d-1}."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")


def loss_oracle(A, xs, iters, gx, glam):
    r = oracle.hopm(A, xs, iters)
    assert r["status"] == 0
    return glam * r["lam"] + sum(float(np.dot(g, x)) for g, x in zip(gx, r["x"]))


@pytest.mark.parametrize("dims,iters", [((4, 5, 3), 3), ((6, 4), 4), ((3, 4, 2, 3), 2), ((5, 3, 4), 1)])
def test_hopm_backward_fd(dims, iters):
    A = synth.tensor("u64", 3, dims)
    xs = [synth.vector("u64", 4, 70 + m, n) + 1.5 for m, n in enumerate(dims)]
    xs = [v / np.linalg.norm(v) for v in xs]
    gx = [synth.vector("u64", 5, 80 + m, n) for m, n in enumerate(dims)]
    glam = 0.7
    gA, gstart = tg.hopm_backward(gu.to_dev(A), [gu.to_dev(v) for v in xs], iters, [gu.to_dev(g) for g in gx],
                                  torch.tensor([glam], dtype=torch.float64))
    torch.cuda.synchronize()
    gA = gA.cpu().numpy()
    h = 1e-6
    flat = A.ravel()
    rng = np.random.default_rng(0)
    for f in rng.choice(flat.size, size=min(8, flat.size), replace=False):
        Ap, Am = flat.copy(), flat.copy()
        Ap[f] += h
        Am[f] -= h
        fd = (loss_oracle(Ap.reshape(dims), xs, iters, gx, glam) - loss_oracle(Am.reshape(dims), xs, iters, gx, glam)) / (2 * h)
        assert abs(fd - gA.ravel()[f]) <= 1e-6 * max(1.0, abs(fd)), (f, fd, gA.ravel()[f])
    for m in range(1, len(dims)):
        g = gstart[m].cpu().numpy()
        for i in range(dims[m]):
            xp = [v.copy() for v in xs]
            xm = [v.copy() for v in xs]
            xp[m][i] += h
            xm[m][i] -= h
            fd = (loss_oracle(A, xp, iters, gx, glam) - loss_oracle(A, xm, iters, gx, glam)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (m, i, fd, g[i])
    assert float(gstart[0].abs().max()) == 0.0


def test_hopm_backward_envelope_at_fixed_point():
    dims = (12, 10, 9)
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    A = synth.tensor("planted", 0, dims, us=us)
    xs = [torch.full((n,), 1.0 / math.sqrt(n), dtype=torch.float64, device=gu.DEV) for n in dims]
    At = gu.to_dev(A)
    r = tg.hopm(At, xs, 40)
    gA, _ = tg.hopm_backward(At, xs, 40, None, torch.tensor([1.0], dtype=torch.float64))
    outer = torch.einsum("i,j,k->ijk", *r.x)
    err = float((gA - outer).norm() / outer.norm())
    assert err <= 1e-8, err


def test_hopm_autograd_matches_backward():
    dims = (5, 6, 4)
    A = gu.to_dev(synth.tensor("u64", 9, dims)).requires_grad_(True)
    xs = [torch.full((n,), 1.0 / math.sqrt(n), dtype=torch.float64, device=gu.DEV).requires_grad_(True) for n in dims]
    out = tg.hopm_autograd(A, xs, 3)
    lam, x = out[0], out[1:]
    L = 2.0 * lam.sum() + sum((xi * (i + 1)).sum() for i, xi in enumerate(x))
    gA, g1 = torch.autograd.grad(L, (A, xs[1]))
    gA2, gs = tg.hopm_backward(A.detach(), [v.detach() for v in xs], 3,
                               [torch.full_like(xi, float(i + 1)) for i, xi in enumerate(x)],
                               torch.tensor([2.0], dtype=torch.float64))
    assert torch.allclose(gA, gA2, rtol=1e-13, atol=1e-15)
    assert torch.allclose(g1, gs[1], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("code", [oracle.F32, oracle.BF16, oracle.E4M3, oracle.F16],
                         ids=["f32", "bf16", "e4m3", "f16"])
def test_hopm_backward_low_precision_fd(code):
    """FP32-vector HOPM backward (binary32 or narrow storage, FP32
    arithmetic) against central finite differences of the FP64 oracle's
    power method on the stored (dequantised) values: the gradient with
    respect to those values, to the accuracy of FP32 accumulation."""
    dims, iters = (6, 5, 4), 3
    A, Ao, scales = gu.inputs(dims, code, seed=4)
    vals = Ao.astype(np.float64) if scales is None else oracle.dequantise(Ao, scales)
    xs = [synth.vector("u64", 4, 70 + m, n) + 1.5 for m, n in enumerate(dims)]
    xs = [(v / np.linalg.norm(v)).astype(np.float32).astype(np.float64) for v in xs]
    gx = [synth.vector("u32", 5, 80 + m, n).astype(np.float64) for m, n in enumerate(dims)]
    glam = 0.7
    f32 = lambda v: torch.from_numpy(np.asarray(v, dtype=np.float32)).to(gu.DEV)  # noqa: E731
    gA, gstart = tg.hopm_backward(gu.to_dev(A), [f32(v) for v in xs], iters, [f32(g) for g in gx],
                                  torch.tensor([glam], dtype=torch.float64),
                                  scales=gu.to_dev(scales) if scales is not None else None, shape=dims)
    torch.cuda.synchronize()
    gA = gA.cpu().numpy().astype(np.float64).ravel()
    h = 1e-6 * float(np.max(np.abs(vals)))
    flat = vals.ravel()
    fds = []
    for f in range(flat.size):
        Ap, Am = flat.copy(), flat.copy()
        Ap[f] += h
        Am[f] -= h
        fds.append((loss_oracle(Ap.reshape(dims), xs, iters, gx, glam)
                    - loss_oracle(Am.reshape(dims), xs, iters, gx, glam)) / (2 * h))
    fds = np.array(fds)
    assert gu.rel_l2(gA, fds) <= 1e-4, gu.rel_l2(gA, fds)
    for m in range(1, len(dims)):
        g = gstart[m].cpu().numpy().astype(np.float64)
        fd = []
        for i in range(dims[m]):
            xp = [v.copy() for v in xs]
            xm = [v.copy() for v in xs]
            xp[m][i] += 1e-6
            xm[m][i] -= 1e-6
            fd.append((loss_oracle(vals, xp, iters, gx, glam) - loss_oracle(vals, xm, iters, gx, glam)) / 2e-6)
        assert gu.rel_l2(g, np.array(fd)) <= 1e-4, (m, gu.rel_l2(g, np.array(fd)))
