"""Helpers shared by the GPU parity tests (inputs, oracle sampling, norms)."""
import numpy as np
import torch

import oracle
import synth

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

TOL = {oracle.F64: 1e-12, oracle.F32: 1e-5, oracle.BF16: 1e-5, oracle.E4M3: 1e-5, oracle.F16: 1e-5}

# Elementwise error model of the FP64 contraction (products in float-float
# pieces on the FP32 pipe, compensated FP32 pairs folded into an FP64 sum
# every 64 products): |y - y_exact| <= F64_MODEL_C * 2^-46 * sum_j |a_j x_j|
# + (ceil(n_k / 64) - 1) * 2^-53 * sum_j |a_j x_j| (the FP64 sum of the folded
# blocks), with y_exact the exactly rounded result.
F64_MODEL_C = 4.0


def f64_model_bound(mag, nk):
    """Largest error the FP64 error model allows for outputs whose
    sum_j |a_j x_j| is `mag`, with n_k terms per output."""
    blocks = max(1, -(-int(nk) // 64))
    return (F64_MODEL_C * 2.0 ** -46 + (blocks - 1) * 2.0 ** -53) * np.asarray(mag, dtype=np.float64)


def rel_l2(got, ref):
    """||got - ref||_2 / ||ref||_2, evaluated with both scaled by max|ref|
    so that huge or tiny magnitudes neither overflow nor underflow."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    m = np.max(np.abs(ref)) if ref.size else 0.0
    if not np.isfinite(m) or not np.all(np.isfinite(got)):
        return float("inf")
    if m == 0.0:
        return float(np.max(np.abs(got))) if got.size else 0.0
    den = np.linalg.norm(ref / m)
    return float(np.linalg.norm(got / m - ref / m) / den)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def inputs(dims, code, seed=0):
    """(A as stored for the GPU, A for the oracle, scales or None, x factory).
    F64: uniform doubles; F32: uniform binary32; BF16/E4M3/F16: N(0,1)exp(U[-3,3])
    binary32 values quantised per slab by the oracle's quantiser."""
    if code == oracle.F64:
        A = synth.tensor("u64", seed, dims)
        return A, A, None
    if code == oracle.F32:
        A = synth.tensor("u32", seed, dims)
        return A, A, None
    src = synth.tensor("lognormal", seed, dims).astype(np.float32)
    codes, scales = oracle.quantise(src, code)
    return codes, codes, scales


def vec(code, n, sid, seed=1):
    if code == oracle.F64:
        return synth.vector("u64", seed, sid, n)
    return synth.vector("u32", seed, sid, n)


def gpu_tvc(tg, A, mode, x, scales=None, **kw):
    At = to_dev(A)
    xt = to_dev(x)
    st = to_dev(scales) if scales is not None else None
    y = tg.tvc(At, mode, xt, scales=st, shape=A.shape, **kw)
    return y.cpu().numpy()


def sample_outputs(dims, mode, count, rng):
    u = int(np.prod(dims[:mode], dtype=np.int64))
    v = int(np.prod(dims[mode + 1:], dtype=np.int64))
    uv = u * v
    picks = rng.integers(0, uv, size=count, dtype=np.int64)
    picks = np.unique(np.concatenate([picks, [0, uv - 1]]))
    return picks, u, v


def oracle_at(kind, seed, dims, mode, x, picks, v, exact=False):
    """Oracle values of y at flat output indices `picks`, from host-generated
    elements A[(i*n_k + j)*v + l] (a dot product per output; with `exact`
    the compensated oracle contraction, the exact sum rounded about once),
    and sum_j |a_j x_j| per output."""
    nk = dims[mode]
    out = np.empty(len(picks))
    mag = np.empty(len(picks))
    j = np.arange(nk, dtype=np.int64)
    for t, o in enumerate(picks):
        i, l = divmod(int(o), v)
        idx = ((i * nk + j) * v + l).astype(np.uint64)
        if kind == "u64":
            a = synth.uniform_f64(seed, synth.STREAM_A, idx)
        else:
            a = synth.uniform_f32(seed, synth.STREAM_A, idx)
        out[t] = oracle.tvc_exact(a, 0, x) if exact else oracle.tvc(a, 0, x)
        mag[t] = np.sum(np.abs(a.astype(np.float64) * x))
    return out, mag
