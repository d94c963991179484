"""Property tests of the oracle over random small shapes (hypothesis): the
TVC, TMC and MTTKRP against numpy's tensordot / einsum for any order, mode
and sizes, and the Khatri-Rao product against Kronecker products."""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

shapes = st.lists(st.integers(1, 5), min_size=1, max_size=5)


def _rand(rng, shape):
    return rng.uniform(-1.0, 1.0, size=shape)


@settings(max_examples=60, deadline=None)
@given(dims=shapes, seed=st.integers(0, 2**31 - 1), data=st.data())
def test_tvc_and_tmc_any_shape(dims, seed, data):
    rng = np.random.default_rng(seed)
    A = _rand(rng, dims)
    k = data.draw(st.integers(0, len(dims) - 1))
    x = _rand(rng, dims[k])
    np.testing.assert_allclose(oracle.tvc(A, k, x), np.tensordot(A, x, axes=([k], [0])), rtol=1e-12, atol=1e-13)
    R = data.draw(st.integers(1, 4))
    X = _rand(rng, (R, dims[k]))
    want = np.moveaxis(np.tensordot(A, X, axes=([k], [1])), -1, k)
    np.testing.assert_allclose(oracle.tmc(A, k, X), want, rtol=1e-12, atol=1e-13)


@settings(max_examples=60, deadline=None)
@given(dims=shapes, seed=st.integers(0, 2**31 - 1), data=st.data())
def test_mttkrp_any_shape(dims, seed, data):
    rng = np.random.default_rng(seed)
    A = _rand(rng, dims)
    d = len(dims)
    k = data.draw(st.integers(0, d - 1))
    R = data.draw(st.integers(1, 3))
    X = [_rand(rng, (n, R)) for n in dims]
    letters = "abcdefg"[:d]
    if d == 1:
        want = np.repeat(A[:, None], R, axis=1)
    else:
        spec = letters + "," + ",".join(f"{letters[m]}z" for m in range(d) if m != k) + "->" + letters[k] + "z"
        want = np.einsum(spec, A, *[X[m] for m in range(d) if m != k])
    got = oracle.mttkrp(A, k, [None if m == k else X[m] for m in range(d)], R=R)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


@settings(max_examples=40, deadline=None)
@given(rows=st.lists(st.integers(1, 4), min_size=1, max_size=4), R=st.integers(1, 4), seed=st.integers(0, 2**31 - 1))
def test_khatri_rao_any_shape(rows, R, seed):
    rng = np.random.default_rng(seed)
    mats = [_rand(rng, (n, R)) for n in rows]
    K = oracle.khatri_rao(mats)
    for r in range(R):
        col = mats[0][:, r]
        for U in mats[1:]:
            col = np.kron(col, U[:, r])
        np.testing.assert_allclose(K[:, r], col, rtol=1e-14, atol=0)
