"""Pins of the FP64 oracle against things other than itself: closed forms,
brute-force unfolding, library routines (numpy einsum / SVD, torch dtype
conversions), invariances, Eq. 3's touched-memory model, the contraction
count of Algorithm 1 and the paper's Table 1.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from tests.conftest import golden

RNG_SEED = 0


def rand_tensor(dims, sid=0, seed=RNG_SEED):
    return synth.tensor("u64", seed, dims, sid)


SHAPES = [(7,), (5, 3), (1, 4), (4, 1), (3, 1, 5), (2, 3, 4), (6, 5, 4, 3), (2, 1, 3, 1, 2),
          (3, 2, 2, 3, 2, 2), (2, 2, 2, 2, 2, 2, 2, 3)]


# ------------------------------------------------------------------ TVC ----

@pytest.mark.parametrize("dims", SHAPES)
def test_tvc_matches_einsum_every_mode(dims):
    A = rand_tensor(dims)
    for k, n in enumerate(dims):
        x = synth.vector("u64", 1, synth.stream_x(k), n)
        want = np.tensordot(A, x, axes=([k], [0]))
        got = oracle.tvc(A, k, x)
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def _unfold(A, k):
    """Mode-k unfolding by explicit index arithmetic: row j = n_k index,
    column = the other indices in row-major order (a brute-force route)."""
    dims = A.shape
    others = [i for i in range(len(dims)) if i != k]
    cols = list(itertools.product(*[range(dims[i]) for i in others]))
    M = [[0.0] * len(cols) for _ in range(dims[k])]
    for j in range(dims[k]):
        for c, idx in enumerate(cols):
            full = list(idx[:k]) + [j] + list(idx[k:])
            M[j][c] = float(A[tuple(full)])
    return M, cols


@pytest.mark.parametrize("dims", [(2, 3, 4), (3, 1, 2, 2), (5, 2)])
def test_tvc_brute_force_unfolding(dims):
    A = rand_tensor(dims, sid=3)
    for k, n in enumerate(dims):
        x = synth.vector("u64", 2, synth.stream_x(k), n)
        M, cols = _unfold(A, k)
        want = [sum(M[j][c] * float(x[j]) for j in range(n)) for c in range(len(cols))]
        got = oracle.tvc(A, k, x).ravel()
        np.testing.assert_allclose(got, np.array(want), rtol=1e-14, atol=1e-15)


def test_tvc_rank1_closed_form():
    dims = (4, 5, 6, 3)
    us = [synth.vector("u64", 5, 30 + j, n) for j, n in enumerate(dims)]
    A = np.einsum("i,j,k,l->ijkl", *us)
    for k in range(4):
        x = synth.vector("u64", 6, synth.stream_x(k), dims[k])
        rest = [us[j] for j in range(4) if j != k]
        want = float(np.dot(us[k], x)) * np.einsum("i,j,k->ijk", *rest)
        np.testing.assert_allclose(oracle.tvc(A, k, x), want, rtol=1e-13, atol=1e-15)


def test_tvc_matrix_cases():
    A = rand_tensor((9, 13))
    x1 = synth.vector("u64", 1, 1, 13)
    x0 = synth.vector("u64", 1, 2, 9)
    np.testing.assert_allclose(oracle.tvc(A, 1, x1), A @ x1, rtol=1e-13)
    np.testing.assert_allclose(oracle.tvc(A, 0, x0), A.T @ x0, rtol=1e-13)


def test_tvc_mode_permutation_invariance():
    dims = (3, 4, 5, 2)
    A = rand_tensor(dims)
    for perm in itertools.permutations(range(4)):
        B = np.ascontiguousarray(np.transpose(A, perm))
        for k in range(4):
            x = synth.vector("u64", 9, 40 + k, dims[k])
            yA = oracle.tvc(A, k, x)
            kb = perm.index(k)
            yB = oracle.tvc(B, kb, x)
            rest = [p for p in perm if p != k]
            order = [sorted(rest).index(p) for p in rest]
            np.testing.assert_allclose(yB, np.transpose(yA, order), rtol=1e-13, atol=1e-15)


def test_tvc_integer_inputs_exact():
    dims = (3, 4, 5)
    rng = np.random.default_rng(3)
    Ai = rng.integers(-1000, 1000, size=dims)
    A = Ai.astype(np.float64)
    for k in range(3):
        xi = rng.integers(-1000, 1000, size=dims[k])
        want = np.tensordot(Ai, xi, axes=([k], [0]))  # exact int64 arithmetic
        got = oracle.tvc(A, k, xi.astype(np.float64))
        assert np.array_equal(got, want.astype(np.float64))


def test_tvc_linearity_ones_and_alpha_beta():
    dims = (4, 6, 5)
    A = rand_tensor(dims)
    for k in range(3):
        x = synth.vector("u64", 3, 1, dims[k])
        z = synth.vector("u64", 3, 2, dims[k])
        np.testing.assert_allclose(oracle.tvc(A, k, 2.0 * x - 3.0 * z),
                                   2.0 * oracle.tvc(A, k, x) - 3.0 * oracle.tvc(A, k, z),
                                   rtol=1e-12, atol=1e-13)
        ones = np.ones(dims[k])
        assert abs(oracle.tvc(A, k, ones).sum() - A.sum()) < 1e-12
        y0 = synth.tensor("u64", 4, [n for i, n in enumerate(dims) if i != k])
        got = oracle.tvc(A, k, x, y=y0, alpha=0.5, beta=-2.0)
        np.testing.assert_allclose(got, 0.5 * oracle.tvc(A, k, x) - 2.0 * y0, rtol=1e-13, atol=1e-14)
        # beta == 0 never reads y (NaN in y is ignored)
        ynan = np.full_like(y0, np.nan)
        assert np.all(np.isfinite(oracle.tvc(A, k, x, y=ynan, alpha=1.0, beta=0.0)))


def test_tvc_successive_contractions_commute():
    dims = (3, 4, 5)
    A = rand_tensor(dims)
    x0, x2 = synth.vector("u64", 1, 1, 3), synth.vector("u64", 1, 3, 5)
    a = oracle.tvc(oracle.tvc(A, 0, x0), 1, x2)
    b = oracle.tvc(oracle.tvc(A, 2, x2), 0, x0)
    np.testing.assert_allclose(a, b, rtol=1e-13)


def test_tvc_narrow_types_dequantise():
    dims = (3, 4, 5)
    src = synth.tensor("lognormal", 0, dims).astype(np.float32)
    for fmt in (oracle.BF16, oracle.E4M3):
        codes, scales = oracle.quantise(src, fmt)
        deq = oracle.dequantise(codes, scales)
        for k in range(3):
            x = synth.vector("u64", 1, 1, dims[k])
            np.testing.assert_allclose(oracle.tvc(codes, k, x, scales=scales),
                                       np.tensordot(deq, x, axes=([k], [0])), rtol=1e-13, atol=1e-13)
    A32 = synth.tensor("u32", 0, dims)
    x = synth.vector("u64", 1, 1, 4)
    np.testing.assert_allclose(oracle.tvc(A32, 1, x),
                               np.tensordot(A32.astype(np.float64), x, axes=([1], [0])), rtol=1e-13)


def _cancelling(dims, mode, seed, kappa=1e6):
    """Uniform A and x, with the last slice of mode `mode` set so that every
    output is about sum|a x| / kappa (heavy cancellation)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, dims)
    x = rng.uniform(-1, 1, dims[mode])
    x[-1] = 0.75
    u, nk = int(np.prod(dims[:mode])), dims[mode]
    Ar = A.reshape(u, nk, -1)
    part = np.einsum("ijl,j->il", Ar[:, :-1, :], x[:-1])
    mag = np.einsum("ijl,j->il", np.abs(Ar[:, :-1, :]), np.abs(x[:-1]))
    Ar[:, -1, :] = -(part - mag / kappa * rng.uniform(-1, 1, part.shape)) / x[-1]
    return A, x


def _exact_fraction(A, mode, x):
    from fractions import Fraction
    u, nk = int(np.prod(A.shape[:mode])), A.shape[mode]
    Ar = A.reshape(u, nk, -1)
    out = np.empty((u, Ar.shape[2]))
    for i in range(u):
        for l in range(Ar.shape[2]):
            out[i, l] = float(sum(Fraction(float(Ar[i, j, l])) * Fraction(float(x[j])) for j in range(nk)))
    return out


@pytest.mark.parametrize("dims", [(4, 7, 5), (3, 40), (2, 3, 33, 2)], ids=lambda d: "x".join(map(str, d)))
def test_tvc_exact_matches_rational_arithmetic_on_cancelling_sums(dims):
    """The compensated oracle contraction against exact rational arithmetic
    (Fraction sums of exact products, rounded once) on sums that cancel to
    about 1e-6 of sum|a x|: within one rounding of the exact value, where the
    plain FP64 sum (and a compensated sum that drops the product errors
    or the addition errors) is off by far more."""
    for k in range(len(dims)):
        A, x = _cancelling(dims, k, seed=3 + k)
        exact = _exact_fraction(A, k, x)
        got = oracle.tvc_exact(A, k, x).reshape(exact.shape)
        assert np.all(np.abs(got - exact) <= 2.0 ** -52 * np.abs(exact)), (dims, k)
        plain = oracle.tvc(A, k, x).reshape(exact.shape)
        assert np.max(np.abs(plain - exact) / np.abs(exact)) > 2.0 ** -45  # the plain sum really errs here


def test_tvc_exact_integer_and_narrow_inputs():
    rng = np.random.default_rng(5)
    A = rng.integers(-1000, 1000, size=(6, 5, 7)).astype(np.float64)
    for k in range(3):
        x = rng.integers(-1000, 1000, size=A.shape[k]).astype(np.float64)
        assert np.array_equal(oracle.tvc_exact(A, k, x), oracle.tvc(A, k, x))
    src = synth.tensor("lognormal", 1, (3, 20, 9)).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.E4M3)
    vals = oracle.dequantise(codes, scales)
    for k in range(3):
        x = synth.vector("u64", 2, synth.stream_x(k), vals.shape[k])
        got = oracle.tvc_exact(codes, k, x, scales=scales)
        exact = _exact_fraction(vals, k, x).reshape(got.shape)
        assert np.all(np.abs(got - exact) <= 2.0 ** -52 * np.abs(exact) + 1e-300)


def test_tvc_bad_arguments():
    A = rand_tensor((2, 3))
    with pytest.raises(ValueError):
        oracle.tvc(A, 2, np.ones(3))
    with pytest.raises(ValueError):
        oracle.tvc(A, 0, np.ones(3))


# ------------------------------------------------------------------ TMC ----

def _tmc_ref(A, k, X):
    """Mode-k product with a matrix through numpy's tensordot: contract the
    n_k axis of A with the columns of X, then move the new R axis to k."""
    return np.moveaxis(np.tensordot(A, X, axes=([k], [1])), -1, k)


@pytest.mark.parametrize("dims", SHAPES)
def test_tmc_matches_tensordot_every_mode(dims):
    A = rand_tensor(dims)
    for k, n in enumerate(dims):
        for R in (1, 3, 8):
            X = synth.tensor("u64", 2, (R, n), synth.stream_x(k))
            got = oracle.tmc(A, k, X)
            want = _tmc_ref(A, k, X)
            assert got.shape == want.shape == tuple(R if i == k else m for i, m in enumerate(dims))
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_tmc_selection_matrices_gather_slices_exactly():
    """A 0/1 matrix whose row r selects index pi(r) of mode k makes the
    product a gather of slices: exact, and a transposed use of X fails."""
    dims = (3, 5, 4, 2)
    A = rand_tensor(dims, sid=4)
    for k, n in enumerate(dims):
        rng = np.random.default_rng(10 + k)
        for R in (n, 2 * n + 1, 1):
            pi = rng.integers(0, n, size=R) if R != n else rng.permutation(n)
            X = np.zeros((R, n))
            X[np.arange(R), pi] = 1.0
            assert np.array_equal(oracle.tmc(A, k, X), np.take(A, pi, axis=k))


def test_tmc_rank1_closed_form():
    dims = (4, 5, 6, 3)
    us = [synth.vector("u64", 5, 30 + j, n) for j, n in enumerate(dims)]
    A = np.einsum("i,j,k,l->ijkl", *us)
    for k in range(4):
        X = synth.tensor("u64", 6, (5, dims[k]), synth.stream_x(k))
        factors = [X @ us[k] if j == k else us[j] for j in range(4)]
        want = np.einsum("i,j,k,l->ijkl", *factors)
        np.testing.assert_allclose(oracle.tmc(A, k, X), want, rtol=1e-13, atol=1e-15)


def test_tmc_matrix_and_vector_cases():
    A = rand_tensor((9, 13))
    X1 = synth.tensor("u64", 1, (4, 13), 1)
    X0 = synth.tensor("u64", 1, (6, 9), 2)
    np.testing.assert_allclose(oracle.tmc(A, 1, X1), A @ X1.T, rtol=1e-13)
    np.testing.assert_allclose(oracle.tmc(A, 0, X0), X0 @ A, rtol=1e-13)
    a = synth.vector("u64", 3, 3, 11)
    Xa = synth.tensor("u64", 3, (5, 11), 4)
    np.testing.assert_allclose(oracle.tmc(a, 0, Xa), Xa @ a, rtol=1e-13)


def test_tmc_rows_are_tvcs_alpha_beta_and_narrow_types():
    dims = (3, 4, 5)
    src = synth.tensor("lognormal", 0, dims).astype(np.float32)
    for k in range(3):
        X = synth.tensor("u64", 7, (3, dims[k]), synth.stream_x(k))
        Y0 = synth.tensor("u64", 8, tuple(3 if i == k else n for i, n in enumerate(dims)))
        for fmt in (oracle.BF16, oracle.E4M3, oracle.F16):
            codes, scales = oracle.quantise(src, fmt)
            deq = oracle.dequantise(codes, scales)
            got = oracle.tmc(codes, k, X, scales=scales, Y=Y0, alpha=-0.5, beta=2.0)
            np.testing.assert_allclose(got, -0.5 * _tmc_ref(deq, k, X) + 2.0 * Y0, rtol=1e-13, atol=1e-13)
            for r in range(3):
                np.testing.assert_array_equal(np.take(oracle.tmc(codes, k, X, scales=scales), r, axis=k),
                                              oracle.tvc(codes, k, X[r], scales=scales))


def test_tmc_bad_arguments():
    A = rand_tensor((2, 3))
    with pytest.raises(ValueError):
        oracle.tmc(A, 1, np.ones((2, 2)))
    with pytest.raises(ValueError):
        oracle.tmc(A, 2, np.ones((2, 3)))
    with pytest.raises(ValueError):
        oracle.tmc(A, 0, np.ones(2))


# -------------------------------------------------- Khatri-Rao, MTTKRP ----

def test_khatri_rao_columns_are_kronecker_products_and_gram_identity():
    U = synth.tensor("u64", 1, (3, 4), 1)
    V = synth.tensor("u64", 1, (5, 4), 2)
    W = synth.tensor("u64", 1, (2, 4), 3)
    K = oracle.khatri_rao([U, V])
    assert K.shape == (15, 4)
    for r in range(4):
        np.testing.assert_array_equal(K[:, r], np.kron(U[:, r], V[:, r]))
    # (U (.) V)^T (U (.) V) = (U^T U) * (V^T V), Hadamard product of the Grams
    np.testing.assert_allclose(K.T @ K, (U.T @ U) * (V.T @ V), rtol=1e-13)
    # associativity, and a single matrix is itself
    np.testing.assert_allclose(oracle.khatri_rao([U, V, W]), oracle.khatri_rao([K, W]), rtol=1e-15)
    np.testing.assert_array_equal(oracle.khatri_rao([W]), W)


@pytest.mark.parametrize("dims", [(7,), (5, 6), (3, 4, 5), (2, 3, 4, 3), (3, 1, 2, 2, 3)])
def test_mttkrp_matches_einsum_every_mode(dims):
    A = rand_tensor(dims, sid=5)
    d = len(dims)
    letters = "abcdefgh"[:d]
    for k in range(d):
        for R in (1, 3):
            X = [synth.tensor("u64", 2, (n, R), 10 + m) for m, n in enumerate(dims)]
            spec = letters + "," + ",".join(f"{letters[m]}z" for m in range(d) if m != k) + "->" + letters[k] + "z"
            want = np.einsum(spec, A, *[X[m] for m in range(d) if m != k]) if d > 1 else A[:, None] * np.ones((1, R))
            got = oracle.mttkrp(A, k, [None if m == k else X[m] for m in range(d)], R=R)
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_mttkrp_one_column_is_the_all_but_one_contraction():
    """R = 1: the contraction of every mode but k with the factor columns,
    done as successive TVCs (highest mode first)."""
    dims = (4, 3, 5, 2)
    A = rand_tensor(dims, sid=6)
    xs = [synth.vector("u64", 3, 20 + m, n) for m, n in enumerate(dims)]
    for k in range(4):
        T = A
        for m in reversed(range(4)):
            if m != k:
                T = oracle.tvc(T, m, xs[m])
        got = oracle.mttkrp(A, k, [x[:, None] for x in xs])
        np.testing.assert_allclose(got[:, 0], T, rtol=1e-13)


def test_mttkrp_rank1_closed_form_and_matrix_case():
    dims = (4, 5, 6)
    us = [synth.vector("u64", 5, 30 + j, n) for j, n in enumerate(dims)]
    A = np.einsum("i,j,k->ijk", *us)
    X = [synth.tensor("u64", 4, (n, 3), 40 + m) for m, n in enumerate(dims)]
    for k in range(3):
        w = np.ones(3)
        for m in range(3):
            if m != k:
                w = w * (us[m] @ X[m])
        np.testing.assert_allclose(oracle.mttkrp(A, k, X), np.outer(us[k], w), rtol=1e-13)
    B = rand_tensor((7, 9), sid=7)
    Y0 = synth.tensor("u64", 6, (7, 2), 1)
    Y1 = synth.tensor("u64", 6, (9, 2), 2)
    np.testing.assert_allclose(oracle.mttkrp(B, 0, [None, Y1]), B @ Y1, rtol=1e-13)
    np.testing.assert_allclose(oracle.mttkrp(B, 1, [Y0, None]), B.T @ Y0, rtol=1e-13)


# ------------------------------------------------------------ gradients ----

@pytest.mark.parametrize("dims", [(4, 5, 3), (6, 7), (2, 3, 2, 3)])
def test_grad_adjoint_identity_and_fd(dims):
    A = rand_tensor(dims)
    for k in range(len(dims)):
        x = synth.vector("u64", 2, 1, dims[k])
        gy = synth.tensor("u64", 3, [n for i, n in enumerate(dims) if i != k])
        y = oracle.tvc(A, k, x)
        gx = oracle.tvc_grad_x(A, k, gy)
        gA = oracle.tvc_grad_A(dims, k, x, gy)
        lhs = float(np.sum(gy * y))
        assert abs(lhs - float(np.dot(gx, x))) < 1e-12 * max(1.0, abs(lhs))
        assert abs(lhs - float(np.sum(gA * A))) < 1e-12 * max(1.0, abs(lhs))
        # central finite differences of L = <gy, A x_k x> in x and in A
        h = 1e-6
        for j in range(dims[k]):
            e = np.zeros(dims[k]); e[j] = h
            fd = (np.sum(gy * oracle.tvc(A, k, x + e)) - np.sum(gy * oracle.tvc(A, k, x - e))) / (2 * h)
            assert abs(fd - gx[j]) < 1e-7 * max(1.0, abs(gx[j]))
        flat = A.ravel()
        for f in (0, flat.size // 2, flat.size - 1):
            Ap, Am = flat.copy(), flat.copy()
            Ap[f] += h; Am[f] -= h
            fd = (np.sum(gy * oracle.tvc(Ap.reshape(dims), k, x)) -
                  np.sum(gy * oracle.tvc(Am.reshape(dims), k, x))) / (2 * h)
            assert abs(fd - gA.ravel()[f]) < 1e-7


# ------------------------------------------------------------------ HOPM ----

def ones_start(dims):
    return [np.ones(n) / math.sqrt(n) for n in dims]


@pytest.mark.parametrize("fn", [oracle.hopm, oracle.hopm3])
def test_hopm_rank1_converges_in_one_sweep(fn):
    dims = (5, 4, 6, 3)
    us = [synth.vector("u64", 8, 50 + j, n) for j, n in enumerate(dims)]
    A = np.einsum("i,j,k,l->ijkl", *us)
    r = fn(A, ones_start(dims), iters=1)
    assert r["status"] == 0
    lam_true = np.prod([np.linalg.norm(u) for u in us])
    assert abs(r["lam"] - lam_true) < 1e-12 * lam_true
    for xj, u in zip(r["x"], us):
        assert abs(abs(np.dot(xj, u / np.linalg.norm(u))) - 1.0) < 1e-13


@pytest.mark.parametrize("fn", [oracle.hopm, oracle.hopm3])
def test_hopm_matrix_gives_top_singular_value(fn):
    A = rand_tensor((12, 9))
    r = fn(A, ones_start(A.shape), iters=500, tol=1e-15)
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(r["lam"] - s[0]) < 1e-10 * s[0]


@pytest.mark.parametrize("dims", [(6, 5, 4), (4, 3, 5, 3), (3, 3, 2, 3, 2)])
def test_hopm_sigma_non_decreasing_and_hopm3_equal(dims):
    A = rand_tensor(dims)
    a = oracle.hopm(A, ones_start(dims), iters=15)
    b = oracle.hopm3(A, ones_start(dims), iters=15)
    assert np.all(np.diff(a["lam_hist"]) >= -1e-13)
    np.testing.assert_allclose(a["lam_hist"], b["lam_hist"], rtol=1e-12)
    for xa, xb in zip(a["x"], b["x"]):
        np.testing.assert_allclose(xa, xb, rtol=1e-10, atol=1e-12)
    # lambda equals the full contraction A(x_0, ..., x_{d-1}) at the end of a sweep
    T = A
    for xj in reversed(a["x"]):
        T = np.tensordot(T, xj, axes=([T.ndim - 1], [0]))
    assert abs(float(T) - a["lam"]) < 1e-6 * a["lam"]


def test_hopm_start_x0_unused_and_stopping_rule():
    dims = (4, 5, 3)
    A = rand_tensor(dims)
    s1 = ones_start(dims)
    s2 = [np.full(4, 123.0)] + s1[1:]
    a = oracle.hopm(A, s1, iters=6)
    b = oracle.hopm(A, s2, iters=6)
    np.testing.assert_array_equal(a["lam_hist"], b["lam_hist"])
    r = oracle.hopm(A, s1, iters=1000, tol=1e-6)
    assert r["sweeps"] < 1000
    h = r["lam_hist"]
    assert abs(h[-1] - h[-2]) <= 1e-6 * h[-1]
    assert all(abs(h[t] - h[t - 1]) > 1e-6 * h[t] for t in range(1, len(h) - 1))


def test_hopm_zero_tensor_status():
    A = np.zeros((3, 4))
    r = oracle.hopm(A, ones_start(A.shape), iters=3)
    assert r["status"] == 5


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_algorithm1_contraction_count(d):
    dims = (2,) * d
    A = rand_tensor(dims)
    a = oracle.hopm(A, ones_start(dims), iters=1)
    b = oracle.hopm3(A, ones_start(dims), iters=1)
    assert a["tvcs"] == d * (d - 1)
    assert b["tvcs"] == d * (d - 1) - (d - 1) * (d - 2) // 2


@pytest.mark.parametrize("d,n", [(2, 9), (3, 7), (4, 5), (5, 3)])
def test_eq3_touched_memory_canonical(d, n):
    A = rand_tensor((n,) * d)
    r = oracle.hopm(A, ones_start((n,) * d), iters=2)
    m_seq = n ** d + 2 * sum(n ** k for k in range(2, d)) + (d + 3) * n
    assert list(r["touched"]) == [d * m_seq] * 2


def test_hopm3_streamed_memory_saving_bands():
    for d_s, lo, hi in golden("hopm3_savings.txt"):
        d, lo, hi = int(d_s), float(lo), float(hi)
        n = 64 if d == 3 else 4
        dims = (n,) * d
        A = rand_tensor(dims)
        a = oracle.hopm(A, ones_start(dims), iters=1)
        b = oracle.hopm3(A, ones_start(dims), iters=1)
        ratio = a["touched"][0] / b["touched"][0]
        assert lo <= ratio <= hi, (d, ratio)


# --------------------------------------------------------------- storage ----

def test_e4m3_decode_matches_spec_and_torch():
    torch = pytest.importorskip("torch")
    for code_s, val_s in golden("e4m3_ocp.txt"):
        code = int(code_s, 16)
        got = oracle.decode_e4m3(code)
        if val_s == "nan":
            assert math.isnan(got)
        else:
            assert got == float(val_s) and math.copysign(1, got) == math.copysign(1, float(val_s))
    codes = torch.arange(256, dtype=torch.uint8)
    ref = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    mine = np.array([oracle.decode_e4m3(c) for c in range(256)])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(mine), nan)
    assert np.array_equal(mine[~nan], ref[~nan])


def test_e4m3_encode_matches_torch_rne_and_saturates():
    torch = pytest.importorskip("torch")
    vals = np.concatenate([
        synth.tensor("lognormal", 1, [20000]).astype(np.float32) * 20,
        np.array([0.0, -0.0, 1e-30, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -9 * 1.5, 448.0, 447.0, 464.0,
                  1e6, -1e6, np.inf, -np.inf], dtype=np.float32),
    ]).astype(np.float32)
    # all midpoints between neighbouring E4M3 magnitudes (ties to even)
    grid = np.array([oracle.decode_e4m3(c) for c in range(0x7F)])
    mids = ((grid[:-1] + grid[1:]) / 2).astype(np.float32)
    vals = np.concatenate([vals, mids, -mids])
    mine = np.array([oracle.e4m3_from_f32(v) for v in vals], dtype=np.uint8)
    inr = np.abs(vals) <= 448.0
    ref = torch.from_numpy(vals[inr]).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(mine[inr], ref)
    assert np.all(mine[~inr & (vals > 0)] == 0x7E) and np.all(mine[~inr & (vals < 0)] == 0xFE)
    assert oracle.e4m3_from_f32(float("nan")) == 0x7F


def test_bf16_rne_matches_torch_and_truncation_is_top_half():
    torch = pytest.importorskip("torch")
    vals = np.concatenate([synth.tensor("lognormal", 2, [20000]),
                           synth.tensor("u64", 3, [20000]) * 1e-3]).astype(np.float32)
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    mine = np.array([oracle.bf16_from_f32(v) for v in vals], dtype=np.uint16)
    assert np.array_equal(mine, ref)
    trunc = np.array([oracle.bf16_from_f32(v, truncate=True) for v in vals], dtype=np.uint16)
    assert np.array_equal(trunc, (vals.view(np.uint32) >> 16).astype(np.uint16))


def test_quantise_per_slab_scales():
    dims = (3, 40, 7)
    src = synth.tensor("lognormal", 4, dims).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.E4M3)
    for i in range(3):
        amax = np.float32(np.abs(src[i]).max())
        assert scales[i] == np.float32(amax / np.float32(448.0))
        assert np.abs(codes[i] & 0x7F).max() == 0x7E  # the slab maximum maps to 448
    deq = oracle.dequantise(codes, scales)
    rel = np.abs(deq - src) / np.abs(src)
    # E4M3 has 3 mantissa bits: relative rounding error <= 2^-4 for normal codes
    big = np.abs(src) > scales.reshape(-1, 1, 1) * 2.0 ** -6
    assert rel[big].max() <= 2.0 ** -4 + 1e-7
    codes_b, scales_b = oracle.quantise(src, oracle.BF16)
    assert np.all(scales_b == 1.0)
    assert np.abs(oracle.dequantise(codes_b, scales_b) - src).max() <= np.abs(src).max() * 2.0 ** -8
    zero = np.zeros((2, 3), dtype=np.float32)
    c0, s0 = oracle.quantise(zero, oracle.E4M3)
    assert np.all(s0 == 1.0) and np.all(c0 == 0)


# ----------------------------------------------------------- binary16 (F16)

def test_f16_decode_matches_numpy_for_every_code():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = codes.view(np.float16).astype(np.float64)
    mine = np.array([oracle.decode_f16(c) for c in range(65536)])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(mine), nan)
    assert np.array_equal(mine[~nan], ref[~nan])
    assert np.array_equal(np.signbit(mine[~nan]), np.signbit(ref[~nan]))
    # IEEE 754 anchors: largest finite, smallest normal, smallest subnormal
    assert oracle.decode_f16(0x7BFF) == 65504.0
    assert oracle.decode_f16(0x0400) == 2.0 ** -14
    assert oracle.decode_f16(0x0001) == 2.0 ** -24


def test_f16_encode_matches_numpy_rne_with_ties_subnormals_and_overflow():
    vals = np.concatenate([
        synth.tensor("lognormal", 5, [20000]).astype(np.float32),
        synth.tensor("u64", 6, [20000]).astype(np.float32) * 1e-5,  # subnormal range
        np.array([0.0, -0.0, 65504.0, 65519.0, 65520.0, 65536.0, 1e6, -1e6, np.inf, -np.inf,
                  2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -24, 2049.0, 2051.0, 1e-30], dtype=np.float32),
    ]).astype(np.float32)
    # every midpoint between neighbouring positive binary16 values (ties to even)
    grid = np.arange(0x7C00, dtype=np.uint32).astype(np.uint16).view(np.float16).astype(np.float64)
    mids = ((grid[:-1] + grid[1:]) / 2).astype(np.float32)
    mids = mids[mids.astype(np.float64) == (grid[:-1] + grid[1:]) / 2]  # exactly representable in FP32
    vals = np.concatenate([vals, mids, -mids])
    ref = vals.astype(np.float16).view(np.uint16)
    mine = np.array([oracle.f16_from_f32(v) for v in vals], dtype=np.uint16)
    assert np.array_equal(mine, ref)
    assert oracle.f16_from_f32(float("nan")) & 0x7E00 == 0x7E00


def test_f16_quantise_unit_scales_and_overflow_status():
    src = synth.tensor("lognormal", 7, (4, 30, 9)).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.F16)
    assert codes.dtype == np.float16 and np.all(scales == 1.0)
    assert np.array_equal(codes.view(np.uint16), src.astype(np.float16).view(np.uint16))
    big = src.copy()
    big[2, 5, 3] = 1e5
    with pytest.raises(oracle.OracleError):
        oracle.quantise(big, oracle.F16)
    codes, _ = oracle.quantise(big, oracle.F16, allow_nonfinite=True)
    assert np.isinf(codes[2, 5, 3])


def test_f16_tvc_is_the_tvc_of_the_decoded_values():
    dims = (5, 6, 7)
    src = synth.tensor("lognormal", 8, dims).astype(np.float32)
    codes, scales = oracle.quantise(src, oracle.F16)
    vals = codes.astype(np.float64)
    for k in range(3):
        x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
        ref = np.tensordot(vals, x, axes=([k], [0]))
        assert np.allclose(oracle.tvc(codes, k, x, scales=scales), ref, rtol=1e-13, atol=0)
        assert np.allclose(oracle.tvc(codes, k, x), ref, rtol=1e-13, atol=0)


# ------------------------------------------- distributed byte model (Eq. 4-7)

def _eq_terms(d, n, p):
    """p * m_seq of Eq. 3 and helpers (integers: every term multiplied by p)."""
    m_seq = n ** d + 2 * sum(n ** k for k in range(2, d)) + (d + 3) * n
    return m_seq


def _sum_pow(lo, hi, n):
    return sum(n ** k for k in range(lo, hi + 1))


@pytest.mark.parametrize("d,n", [(2, 6), (3, 6), (3, 12), (4, 6), (5, 4), (6, 4), (10, 4)])
def test_dhopm_byte_model_equations_4_to_7(d, n):
    for p in [q for q in range(1, n + 1) if n % q == 0]:
        m_seq = _eq_terms(d, n, p)
        M = {}
        for s in range(d):
            tot = 0
            for j in range(d):
                got = oracle.dhopm_touched(d, n, p, s, j)
                tot += got
                if j == s:  # Eq. 4 (regular division: the brackets are exact)
                    want_p = n ** d + 2 * _sum_pow(2, d - 1, n) + 4 * n + (d - 1) * n * p
                else:  # Eq. 5, l = 0 for j < s and 1 for j > s
                    l = 0 if j < s else 1
                    want_p = m_seq + (p - 1) * (2 * _sum_pow(2, d - s - l, n) + (d + 2) * n)
                assert got * p == want_p, (d, n, p, s, j, got)
            # Eq. 6: the process's total over the d external iterations
            want_p = (d * m_seq + (p - 1) * (d - 1) * (d + 3) * n
                      + (p - 1) * (s * 2 * _sum_pow(2, d - s, n) + (d - s - 1) * 2 * _sum_pow(2, d - s - 1, n)))
            assert tot * p == want_p, (d, n, p, s)
            M[s] = tot
        for s in range(1, d):  # Eq. 7: the recursion over the split dimension
            assert (M[s - 1] - M[s]) * p == (p - 1) * ((d - s - 1) * 2 * n ** (d - s) + (s - 1) * 2 * n ** (d - s + 1))


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4), (4, 3), (5, 3)])
def test_dhopm_byte_model_one_process_is_the_oracles_own_count(d, n):
    """p = 1: the size-only counter equals the touched counts of the oracle's
    HOPM runs (canonical chain: Eq. 3; three-buffer chain: Algorithm 1)."""
    dims = (n,) * d
    A = rand_tensor(dims)
    a = oracle.hopm(A, ones_start(dims), iters=1)
    b = oracle.hopm3(A, ones_start(dims), iters=1)
    assert sum(oracle.dhopm_touched(d, n, 1, 0, j) for j in range(d)) == a["touched"][0]
    assert sum(oracle.dhopm_touched(d, n, 1, 0, j, three=True) for j in range(d)) == b["touched"][0]
    assert a["touched"][0] == d * _eq_terms(d, n, 1)


def test_dhopm3_saving_is_flat_in_processes_and_split():
    for d_s, n_s, lo_p, hi_p, lo, hi in golden("dhopm_byte_model.txt"):
        d, n, lo, hi = int(d_s), int(n_s), float(lo), float(hi)
        ratios = []
        for p in [q for q in range(1, n + 1) if n % q == 0 and float(lo_p) <= q / n <= float(hi_p)]:
            for s in range(d):
                a = sum(oracle.dhopm_touched(d, n, p, s, j) for j in range(d))
                b = sum(oracle.dhopm_touched(d, n, p, s, j, three=True) for j in range(d))
                ratios.append(a / b)
        assert ratios and lo <= min(ratios) and max(ratios) <= hi, (d, min(ratios), max(ratios))
    # the minimum of about 3.3x for d = 10 sits at p = n (one slab per process)
    assert 3.2 <= min(sum(oracle.dhopm_touched(10, 8, 8, s, j) for j in range(10)) /
                      sum(oracle.dhopm_touched(10, 8, 8, s, j, three=True) for j in range(10))
                      for s in range(10)) <= 3.4


# ------------------------------------------------------------ Jacobi HOPM

def test_jacobi_first_sweep_is_the_einsum_contractions():
    dims = (5, 6, 4)
    A = rand_tensor(dims, sid=3)
    xs = [synth.vector("u64", 9, 30 + m, n) for m, n in enumerate(dims)]
    r = oracle.hopm_jacobi(A, xs, 1)
    zs = [np.einsum("ijk,j,k->i", A, xs[1], xs[2]), np.einsum("ijk,i,k->j", A, xs[0], xs[2]),
          np.einsum("ijk,i,j->k", A, xs[0], xs[1])]
    for got, z in zip(r["x"], zs):
        np.testing.assert_allclose(got, z / np.linalg.norm(z), rtol=1e-13, atol=1e-15)
    assert abs(r["lam"] - np.linalg.norm(zs[2])) <= 1e-13 * np.linalg.norm(zs[2])


def test_jacobi_rank1_in_one_sweep_and_svd_for_order_2():
    us = [synth.vector("u64", 4, 50 + j, n) for j, n in enumerate((6, 5, 7))]
    A = np.einsum("i,j,k->ijk", *us)
    # one sweep aligns every vector with its factor; lambda, formed from the
    # previous sweep's vectors, reaches ||A|| = prod ||u_j|| in the second
    r = oracle.hopm_jacobi(A, ones_start(A.shape), 1)
    for xg, u in zip(r["x"], us):
        assert abs(abs(np.dot(xg, u / np.linalg.norm(u))) - 1) <= 1e-13
    r = oracle.hopm_jacobi(A, ones_start(A.shape), 2)
    assert abs(r["lam"] - np.prod([np.linalg.norm(u) for u in us])) <= 1e-13 * r["lam"]
    M = rand_tensor((9, 7), sid=4)
    r = oracle.hopm_jacobi(M, ones_start(M.shape), 400, 1e-15)
    assert abs(r["lam"] - np.linalg.svd(M, compute_uv=False)[0]) <= 1e-10 * r["lam"]


def test_jacobi_leaves_a_converged_point_fixed():
    dims = (6, 7, 5)
    A = rand_tensor(dims, sid=5)
    gs = oracle.hopm(A, ones_start(dims), 300, 1e-15)
    # near the fixed point both maps move the vectors by the same order as
    # the remaining residual (lambda converges as its square)
    step = max(np.max(np.abs(a - b)) for a, b in zip(oracle.hopm(A, gs["x"], 1)["x"], gs["x"]))
    r = oracle.hopm_jacobi(A, gs["x"], 1)
    assert abs(r["lam"] - gs["lam"]) <= 1e-10 * gs["lam"]
    for a, b in zip(r["x"], gs["x"]):
        assert np.max(np.abs(a - b)) <= 4 * step + 1e-13
