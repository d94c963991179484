"""Writes tests/golden/hopm_fullsize.json: the FP64 oracle's results for the
two full-size power-method workloads, so that GPU tests and the benchmark can
compare against them without re-running a CPU computation of minutes.

Workloads (inputs from the host generator ``synth``; every computation below
is the oracle's, ``oracle.quantise`` and ``oracle.hopm3``, the three-buffer
HOPM of Algorithm 1, itself pinned to the canonical HOPM of Section 3):

* planted: order-4 tensor 256^4 in binary32, A = 10 u_0 o u_1 o u_2 o u_3 +
  0.01 N(0,1), u_j unit Gaussian vectors (synth streams 10 + j, seed 0);
  start x_j = (u_j + g_j) / ||u_j + g_j|| with g_j an independent unit
  Gaussian vector (seed 1, the same streams), rounded to binary32 like the
  start vectors of an FP32 run; 50 sweeps, tol 1e-8.
* mixed: order-3 tensor 2048^3, entries N(0,1) exp(U[-3,3]) rounded to
  binary32 (seed 0, stream 0); the binary32 source itself and its per-slab
  BF16 and E4M3 storage (Section 5.5: low precision for storage only, one
  FP32 scale per 2048 x 2048 slab); 30 sweeps from normalised all-ones
  vectors (1/sqrt(2048) rounded to binary32), tol 0.

Recorded per run: lambda of every sweep, the sweep count, entries of every
final x_j at 16 fixed indices, and for the stored formats the SHA-256 of the
oracle's codes and scales (so a full-size quantiser can be checked bit for
bit).  For the planted run also the subspace error max_j sqrt(1 - <x_j, u_j>^2).

    python tests/golden/make_fullsize_hopm.py [--out PATH] [--threads T]

Needs about 55 GB of host memory and 10-20 minutes on 16 cores.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

PLANTED_DIMS = (256, 256, 256, 256)
MIXED_DIMS = (2048, 2048, 2048)


def probe_indices(n):
    return [int(i) for i in np.unique(np.linspace(0, n - 1, 16).round().astype(np.int64))]


def _lognormal_chunk(lo, hi):
    return lo, synth.lognormal_mix_f64(0, synth.STREAM_A, np.arange(lo, hi, dtype=np.uint64)).astype(np.float32)


def _planted_chunk(lo, hi, dims, us):
    return lo, synth.planted_rank1_f64(0, dims, us, np.arange(lo, hi, dtype=np.int64)).astype(np.float32)


def fill(n, chunk_fn, args, procs, chunk=1 << 22):
    """Elements 0..n-1 of a generator, rounded to binary32 (the rounding the
    device fill applies), computed in chunks by a pool of processes (spawned,
    so no state is inherited)."""
    import multiprocessing as mp
    out = np.empty(n, dtype=np.float32)
    jobs = [(lo, min(n, lo + chunk)) + tuple(args) for lo in range(0, n, chunk)]
    with mp.get_context("spawn").Pool(procs) as pool:
        for lo, vals in pool.starmap(chunk_fn, jobs, chunksize=1):
            out[lo:lo + vals.size] = vals
    return out


def sha(a):
    h = hashlib.sha256()
    flat = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
    step = 1 << 30
    for lo in range(0, flat.size, step):
        h.update(flat[lo:lo + step])
    return h.hexdigest()


def record(res, dims, seconds):
    return {"status": res["status"], "sweeps": res["sweeps"], "lam": res["lam"],
            "lam_hist": [float(v) for v in res["lam_hist"]],
            "x_probe": [{str(i): float(x[i]) for i in probe_indices(len(x))} for x in res["x"]],
            "oracle_seconds": round(seconds, 1)}


def planted_start(dims):
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    xs = []
    for j, n in enumerate(dims):
        v = us[j] + synth.unit_gaussian(1, synth.stream_u(j), n)
        xs.append(f32_start(v / np.linalg.norm(v)))
    return us, xs


def f32_start(v):
    """A start vector as an FP32 power method receives it: rounded to binary32."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "hopm_fullsize.json"))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1, help="generator processes")
    ap.add_argument("--only", choices=["planted", "mixed"], default=None)
    a = ap.parse_args(argv)
    oracle.build()
    out = {"generated_by": "tests/golden/make_fullsize_hopm.py", "oracle": "oracle.hopm3 (FP64)",
           "host_threads": a.threads}
    if os.path.exists(a.out):
        with open(a.out) as fh:
            out.update({k: v for k, v in json.load(fh).items() if k in ("planted", "mixed")})

    if a.only in (None, "planted"):
        dims = PLANTED_DIMS
        us, xs = planted_start(dims)
        t0 = time.time()
        A = fill(math.prod(dims), _planted_chunk, (dims, us), a.threads).reshape(dims)
        print(f"planted tensor generated in {time.time() - t0:.0f} s", flush=True)
        t0 = time.time()
        res = oracle.hopm3(A, xs, 50, 1e-8)
        sec = time.time() - t0
        rec = record(res, dims, sec)
        rec["subspace_error"] = max(math.sqrt(max(0.0, 1.0 - float(np.dot(x, u)) ** 2))
                                    for x, u in zip(res["x"], us))
        rec.update(dims=list(dims), iters=50, tol=1e-8, start="(u_j + g_j)/||.||, g_j unit Gaussian seed 1")
        out["planted"] = rec
        print(f"planted: lambda {res['lam']:.12g} after {res['sweeps']} sweeps ({sec:.0f} s)", flush=True)
        del A

    if a.only in (None, "mixed"):
        dims = MIXED_DIMS
        t0 = time.time()
        src = fill(math.prod(dims), _lognormal_chunk, (), a.threads).reshape(dims)
        print(f"mixed source generated in {time.time() - t0:.0f} s", flush=True)
        ones = [f32_start(np.full(n, 1.0 / math.sqrt(n))) for n in dims]
        mixed = {"dims": list(dims), "iters": 30, "tol": 0.0, "start": "normalised all-ones"}
        t0 = time.time()
        res = oracle.hopm3(src, ones, 30)
        mixed["f32"] = record(res, dims, time.time() - t0)
        print(f"mixed f32: lambda {res['lam']:.12g} ({time.time() - t0:.0f} s)", flush=True)
        for name, fmt in (("bf16", oracle.BF16), ("e4m3", oracle.E4M3)):
            t0 = time.time()
            codes, scales = oracle.quantise(src, fmt)
            tq = time.time() - t0
            t0 = time.time()
            res = oracle.hopm3(codes, ones, 30, scales=scales)
            rec = record(res, dims, time.time() - t0)
            rec.update(sha256_codes=sha(codes), sha256_scales=sha(scales), quantise_seconds=round(tq, 1))
            mixed[name] = rec
            print(f"mixed {name}: lambda {res['lam']:.12g} ({rec['oracle_seconds']} s)", flush=True)
            del codes, scales
        out["mixed"] = mixed
        del src

    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print("wrote", a.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
