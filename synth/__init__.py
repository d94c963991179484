"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the tensor-vector contraction or of the
power method: it only turns (seed, stream, element index) into numbers.
Everything is counter based, so any element of any tensor can be produced on
its own (random access), which is what the sampled full-size parity checks
need, and the device-side fill kernels in ``synth/csrc`` reproduce exactly the
same bits (every step below is an exactly rounded IEEE operation or an
integer operation, with no fused multiply-add).

Generator: Philox4x32-10, from its published definition (Salmon, Moraes,
Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
Element ``f`` of stream ``sid`` under ``seed`` uses the counter
``(f mod 2^32, f div 2^32, sid, word3)`` and the key
``(seed mod 2^32, seed div 2^32)``.

Distributions
-------------
* ``uniform_f64``: 53 random bits ``m`` -> ``m * 2^-52 - 1`` in [-1, 1).
* ``uniform_f32``: 24 random bits ``m`` -> ``m * 2^-23 - 1`` in [-1, 1),
  exact in binary32.
* ``gaussian_f64``: Marsaglia's polar method with a logarithm written here
  from its series (``ln_f64``); attempt ``a`` (0..31) uses ``word3 = a``.
* ``lognormal_mix_f64``: ``N(0,1) * exp(U[-3, 3])`` (the wide-dynamic-range
  recipe of the mixed-precision workload); the uniform uses ``word3 = 32``
  and ``exp_f64`` is written here from its Taylor series.
* ``planted_rank1_f64``: ``10 * u0[i0] u1[i1] ... + 0.01 * N(0,1)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10", "uniform_f64", "uniform_f32", "gaussian_f64",
    "lognormal_mix_f64", "planted_rank1_f64", "ln_f64", "exp_f64",
    "tensor", "vector", "STREAM_A", "stream_x", "stream_u", "STREAM_NOISE",
    "stream_batch",
]

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# Stream identifiers used by the workloads (one per independent input).
STREAM_A = 0


def stream_x(k: int) -> int:
    """Stream of the contraction vector for mode ``k``."""
    return 1 + k


def stream_u(j: int) -> int:
    """Stream of the planted factor ``u_j``."""
    return 10 + j


STREAM_NOISE = 20


def stream_batch(b: int) -> int:
    """Stream of tensor ``b`` of a batch."""
    return 1000 + b


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32-valued arrays (held as uint64).

    Returns the four output words.  Each round multiplies words 0 and 2 by
    the two multipliers, xors the high halves into the other words with the
    round key, and permutes; the key is bumped by the Weyl constants between
    rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
    return c0, c1, c2, c3


def _words(seed: int, sid: int, idx, word3: int = 0):
    idx = np.asarray(idx, dtype=np.uint64)
    return philox4x32_10(idx & _MASK, idx >> _S32, np.uint64(sid),
                         np.uint64(word3), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def _u53(w_lo, w_hi):
    m = (w_hi << np.uint64(21)) | (w_lo >> np.uint64(11))
    return m.astype(np.float64) * 2.0 ** -52 - 1.0


def uniform_f64(seed: int, sid: int, idx) -> np.ndarray:
    """Uniform [-1, 1) doubles for element indices ``idx``."""
    w0, w1, _, _ = _words(seed, sid, idx)
    return _u53(w0, w1)


def uniform_f32(seed: int, sid: int, idx) -> np.ndarray:
    """Uniform [-1, 1) binary32 values (24 random bits) for ``idx``."""
    w0, _, _, _ = _words(seed, sid, idx)
    m = (w0 >> np.uint64(8)).astype(np.float64)
    return (m * 2.0 ** -23 - 1.0).astype(np.float32)


_LN2 = 0.6931471805599453          # nearest double to ln 2
_SQRT_HALF = 0.7071067811865476    # nearest double to 1/sqrt(2)


def ln_f64(s) -> np.ndarray:
    """Natural logarithm of positive normal doubles, from the series
    ln m = 2 (t + t^3/3 + t^5/5 + ...), t = (m-1)/(m+1), after the exact
    split s = m 2^e with m in [1/sqrt2, sqrt2).  Plain rounded operations
    only, evaluated in a fixed order (Horner in t^2)."""
    s = np.asarray(s, dtype=np.float64)
    m, e = np.frexp(s)                      # s = m * 2^e, m in [0.5, 1), exact
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    acc = np.full_like(t, 1.0 / 23.0)
    for k in range(10, -1, -1):             # 1/21, 1/19, ..., 1/1
        acc = acc * t2 + 1.0 / (2 * k + 1)
    return e * _LN2 + 2.0 * (t * acc)


def exp_f64(t) -> np.ndarray:
    """exp(t) for |t| <= 4: Taylor series of exp(t/16) to degree 13 (Horner),
    then squared four times.  Plain rounded operations in a fixed order."""
    r = np.asarray(t, dtype=np.float64) / 16.0
    acc = np.full_like(r, 1.0 / 6227020800.0)   # 1/13!
    fact = 6227020800.0
    for k in range(12, -1, -1):
        fact = fact / (k + 1)                   # k! exactly (k <= 12)
        acc = acc * r + 1.0 / fact
    for _ in range(4):
        acc = acc * acc
    return acc


_POLAR_ATTEMPTS = 32


def gaussian_f64(seed: int, sid: int, idx) -> np.ndarray:
    """Standard normal doubles by the polar method; attempt ``a`` draws
    (u, v) from counter word 3 = a; 0.0 if all 32 attempts are rejected."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = np.zeros(idx.shape, dtype=np.float64)
    todo = np.ones(idx.shape, dtype=bool)
    for a in range(_POLAR_ATTEMPTS):
        if not todo.any():
            break
        w0, w1, w2, w3 = _words(seed, sid, idx[todo], a)
        u = _u53(w0, w1)
        v = _u53(w2, w3)
        s = u * u + v * v
        ok = (s > 0.0) & (s < 1.0)
        ss = np.where(ok, s, 0.5)
        z = u * np.sqrt((-2.0 * ln_f64(ss)) / ss)
        sel = np.flatnonzero(todo)
        out[sel[ok]] = z[ok]
        todo[sel[ok]] = False
    return out


def lognormal_mix_f64(seed: int, sid: int, idx) -> np.ndarray:
    """N(0,1) * exp(U[-3, 3]) per element (the uniform from word3 = 32)."""
    idx = np.asarray(idx, dtype=np.uint64)
    g = gaussian_f64(seed, sid, idx)
    w0, w1, _, _ = _words(seed, sid, idx, 32)
    t = 3.0 * _u53(w0, w1)
    return g * exp_f64(t)


def planted_rank1_f64(seed: int, dims, us, idx) -> np.ndarray:
    """10 * u_0[i_0] u_1[i_1] ... u_{d-1}[i_{d-1}] + 0.01 * N(0,1) at flat
    row-major indices ``idx``; ``us`` are the (already normalised) factors.
    The product is formed left to right, 10 * u_0 first."""
    idx = np.asarray(idx, dtype=np.int64)
    dims = [int(n) for n in dims]
    rem = idx.copy()
    digits = []
    for n in reversed(dims):
        digits.append(rem % n)
        rem //= n
    digits.reverse()
    acc = 10.0 * np.asarray(us[0], dtype=np.float64)[digits[0]]
    for j in range(1, len(dims)):
        acc = acc * np.asarray(us[j], dtype=np.float64)[digits[j]]
    z = gaussian_f64(seed, STREAM_NOISE, idx.astype(np.uint64))
    return acc + 0.01 * z


def tensor(kind: str, seed: int, dims, sid: int = STREAM_A, us=None) -> np.ndarray:
    """A whole dense row-major tensor (small sizes only) of the given kind:
    'u64' uniform doubles, 'u32' uniform binary32, 'gauss', 'lognormal',
    'planted'."""
    dims = [int(n) for n in dims]
    n = int(np.prod(dims, dtype=np.int64)) if dims else 1
    idx = np.arange(n, dtype=np.uint64)
    if kind == "u64":
        out = uniform_f64(seed, sid, idx)
    elif kind == "u32":
        out = uniform_f32(seed, sid, idx)
    elif kind == "gauss":
        out = gaussian_f64(seed, sid, idx)
    elif kind == "lognormal":
        out = lognormal_mix_f64(seed, sid, idx)
    elif kind == "planted":
        out = planted_rank1_f64(seed, dims, us, idx)
    else:
        raise ValueError(f"unknown kind {kind!r}")
    return out.reshape(dims)


def vector(kind: str, seed: int, sid: int, n: int) -> np.ndarray:
    """A length-``n`` vector of the given kind (see :func:`tensor`)."""
    return tensor(kind, seed, [n], sid)


def unit_gaussian(seed: int, sid: int, n: int) -> np.ndarray:
    """A Gaussian vector scaled to unit Euclidean norm (planted factors)."""
    g = gaussian_f64(seed, sid, np.arange(n, dtype=np.uint64))
    return g / np.sqrt(np.dot(g, g))
