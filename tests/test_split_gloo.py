"""The N > 1 paths on CPU: two gloo ranks (world size 2, 127.0.0.1).

- The 1D split with real collectives: each rank holds its slab of the
  tensor (the package's partition), contracts it with the oracle, and the
  ranks combine as Section 3.1 and Algorithm 1 prescribe: all-gather of the
  disjoint output slabs (Eq. 1), sum all-reduce of the full-size partials
  (Eq. 2), and in the distributed HOPM an n_j-entry sum all-reduce for
  j != s and a gather of x_s's ranges for j = s.  The combined results must
  equal the oracle on the unsplit tensor.
- bench.py's combination of the replicas' timings (maximum over ranks).
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

WORLD = 2


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab(A, s, a, b):
    return np.take(A, np.arange(a, b), axis=s)


def _all_but(oracle, T, xs, j):
    """Contraction of every mode but j, last mode first (plain oracle TVCs)."""
    for m in reversed(range(T.ndim)):
        if m != j:
            T = oracle.tvc(T, m, xs[m])
    return T


def _check_dtvc(rank, oracle, synth, tg):
    for dims in [(6, 5, 4), (7, 3, 5, 2), (13, 40)]:
        A = synth.tensor("u64", 7, dims)
        for s in range(len(dims)):
            st = tg.split_1d(dims[s], WORLD)
            if len(st) - 1 != WORLD:
                continue
            Ar = _slab(A, s, st[rank], st[rank + 1])
            for k in range(len(dims)):
                x = synth.vector("u64", 1, synth.stream_x(k), dims[k])
                ref = oracle.tvc(A, k, x)
                if k != s:  # Eq. 1: gather the disjoint output slabs
                    mine = oracle.tvc(Ar, k, x)
                    got = [None] * WORLD
                    dist.all_gather_object(got, mine)
                    so = s if s < k else s - 1
                    assert np.array_equal(np.concatenate(got, axis=so), ref)
                else:  # Eq. 2: sum the full-size partials
                    mine = torch.from_numpy(np.ascontiguousarray(oracle.tvc(Ar, k, x[st[rank]:st[rank + 1]])))
                    dist.all_reduce(mine, op=dist.ReduceOp.SUM)
                    tot = mine.numpy()
                    assert np.max(np.abs(tot - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def _check_dhopm(rank, oracle, synth, tg):
    for dims in [(6, 7, 5), (4, 5, 3, 6), (9, 8)]:
        A = synth.tensor("u64", 3, dims)
        d = len(dims)
        iters = 5
        ref = oracle.hopm(A, [np.ones(n) / math.sqrt(n) for n in dims], iters)
        for s in range(d):
            st = tg.split_1d(dims[s], WORLD)
            if len(st) - 1 != WORLD:
                continue
            a, b = st[rank], st[rank + 1]
            Ar = _slab(A, s, a, b)
            x = [np.ones(n) / math.sqrt(n) for n in dims]  # duplicated on every rank
            hist = []
            for _ in range(iters):
                for j in range(d):
                    local = [x[m][a:b] if m == s else x[m] for m in range(d)]
                    z = _all_but(oracle, Ar, local, j)
                    if j != s:  # array reduction of n_j entries
                        t = torch.from_numpy(np.ascontiguousarray(z))
                        dist.all_reduce(t, op=dist.ReduceOp.SUM)
                        z = t.numpy()
                    else:  # array gather of the ranks' ranges
                        got = [None] * WORLD
                        dist.all_gather_object(got, z)
                        z = np.concatenate(got)
                    sigma = float(np.linalg.norm(z))
                    x[j] = z / sigma
                hist.append(sigma)
            np.testing.assert_allclose(hist, ref["lam_hist"], rtol=1e-12)
            for xg, xr in zip(x, ref["x"]):
                assert np.max(np.abs(xg - xr)) <= 1e-12


def _check_bench_max(rank):
    import bench
    got = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    assert got == 10.0 + (WORLD - 1)
    assert bench.max_over_ranks(3.5, None, None) == 3.5


def _worker(rank, port, root):
    import sys
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import oracle
        import synth
        import paper_2501_03121_gb300 as tg
        _check_dtvc(rank, oracle, synth, tg)
        _check_dhopm(rank, oracle, synth, tg)
        _check_bench_max(rank)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_split_and_bench_over_two_gloo_ranks():
    from tests.conftest import ROOT
    from paper_2501_03121_gb300 import build as b
    import oracle
    b.build()
    oracle.build()
    mp.spawn(_worker, args=(_free_port(), ROOT), nprocs=WORLD, join=True)
