"""The 1D split of Section 3.1 on the host: the partition (tvc_split_1d,
through the C ABI; it launches nothing) and the split identities Eq. 1 and
Eq. 2 on the oracle, for every splitting dimension s and contraction mode k.
"""
import numpy as np
import pytest

import oracle
import synth

tg = pytest.importorskip("paper_2501_03121_gb300")


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2501_03121_gb300 import build as b
    b.build()


def test_partition_of_the_papers_example():
    # Fig. 2: A of 2 x 3 x 4 split by p = 3 along s = 0, 1, 2.  Along the
    # last dimension the quotient [4/3] becomes 4/2: only two ranks remain.
    assert tg.split_1d(2, 3) == [0, 1, 2]
    assert tg.split_1d(3, 3) == [0, 1, 2, 3]
    assert tg.split_1d(4, 3) == [0, 2, 4]


def test_partition_invariants():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        n = int(rng.integers(1, 5000))
        p = int(rng.integers(1, 65))
        q = int(rng.choice([1, 2, 4, 8, 16]))
        st = tg.split_1d(n, p, q)
        ranks = len(st) - 1
        assert st[0] == 0 and st[-1] == n
        assert 1 <= ranks <= p
        sizes = np.diff(st)
        assert np.all(sizes > 0)
        chunk = sizes[0]
        # every rank but the last holds one chunk: ceil(n/p) rounded up to q
        assert chunk == -(-(-(-n // p)) // q) * q or ranks == 1
        assert np.all(sizes[:-1] == chunk)
        assert sizes[-1] <= chunk
        assert ranks == -(-n // chunk)


def test_partition_rejects_bad_arguments():
    for n, p, q in ((0, 2, 1), (5, 0, 1), (5, 65, 1), (5, 2, 0)):
        with pytest.raises(ValueError):
            tg.split_1d(n, p, q)


def _slab(A, s, a, b):
    return np.take(A, np.arange(a, b), axis=s)


@pytest.mark.parametrize("dims", [(6, 5, 4), (2, 3, 4), (7, 3, 5, 2), (13, 40)])
def test_split_identities_on_the_oracle(dims):
    A = synth.tensor("u64", 7, dims)
    for s in range(len(dims)):
        for p in (2, 3, 4):
            st = tg.split_1d(dims[s], p)
            for k in range(len(dims)):
                x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
                ref = oracle.tvc(A, k, x)
                if k != s:
                    # Eq. 1: the ranks' outputs are disjoint slabs of Y along s
                    # (s - 1 once mode k < s has been removed); each output is the
                    # same dot product as in the unsplit tensor, so bit-equal.
                    so = s if s < k else s - 1
                    parts = [oracle.tvc(_slab(A, s, st[r], st[r + 1]), k, x) for r in range(len(st) - 1)]
                    assert np.array_equal(np.concatenate(parts, axis=so), ref)
                else:
                    # Eq. 2: full-size partials against the ranks' parts of x, summed
                    parts = [oracle.tvc(_slab(A, s, st[r], st[r + 1]), k, x[st[r]:st[r + 1]])
                             for r in range(len(st) - 1)]
                    tot = np.sum(parts, axis=0)
                    assert tot.shape == ref.shape
                    assert np.max(np.abs(tot - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
