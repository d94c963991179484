"""Benchmark: achieved HBM bandwidth of the mode-oblivious TVC on one GB300.

Workload (one step): the TVC bandwidth sweep, i.e. the contraction along
EVERY mode of the dense row-major tensors 1024^3, 128^4, 40^6 and
65536x16384 (order 2), each stored in FP64 and in FP32, entries uniform
[-1, 1) (counter-based generator, seed 0), x uniform [-1, 1).  30 TVCs per
step, about 380 GB of algorithmic traffic.  value = algorithmic bytes / time
(GB/s), summed over ranks; each rank runs an independent replica (the
single-GPU path has no data-parallel exchange).

Every input is far larger than the 129 MB L2 (the smallest is 1.07 GB), so
no flush is needed between timed iterations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --case tvc|batched ...   (one case, for profiling)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TVC/HOPM achieved HBM GB/s (% of GB300 peak), FP64 vs BF16 at stated error"
TENSORS = [(1024, 1024, 1024), (128, 128, 128, 128), (40, 40, 40, 40, 40, 40), (65536, 16384)]
WORKLOAD = ("TVC bandwidth sweep: every mode of 1024^3, 128^4, 40^6 and 65536x16384, "
            "FP64 and FP32 storage, uniform[-1,1) seed 0")


def tvc_bytes(dims, mode, esize, vsize):
    """Algorithmic bytes of one TVC with beta = 0: read A once, read x,
    write y (N/n_k entries)."""
    N = math.prod(dims)
    return N * esize + dims[mode] * vsize + (N // dims[mode]) * vsize


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record():
    """DRAM traffic of the dominant kernel measured by ncu
    (profiles/roofline_traffic.json), valid only while the kernel's source
    section is unchanged (its hash is recorded with the counters)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        src = open(os.path.join(ROOT, rec["source"])).read()
        a = src.index(rec["section_begin"])
        b = src.index(rec["section_end"], a)
        sha = hashlib.sha256(src[a:b].encode()).hexdigest()[:16]
        return rec if sha == rec["source_sha"] else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        mhz = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def max_over_ranks(value: float, pg, device) -> float:
    """The largest of the ranks' values (the timed region ends with the
    slowest replica); pg is torch.distributed (or None for one rank)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------ CPU-baseline (oracle) leg
#
# The only part of this file that runs the oracle (the FP64 CPU reference
# under oracle/): its timings on the host cores, and the reference values at
# sampled outputs of the timed GPU calls, from which the error of the timed
# results is reported.

class OracleSample:
    """A bounded sample of the sweep workload for the FP64 CPU oracle: each
    tensor cut to its first slabs (dims[0] reduced so the cut holds about
    2^22 elements), in FP64 and FP32 storage, contracted along every mode."""

    def __init__(self, elems=1 << 22):
        import oracle
        import synth
        oracle.build()
        self.oracle = oracle
        self.cut = []
        for dims in TENSORS:
            rest = math.prod(dims[1:])
            n0 = max(1, min(dims[0], elems // rest))
            self.cut.append((n0,) + tuple(dims[1:]))
        self.items = []
        for kind, es in (("u64", 8), ("u32", 4)):
            for sd in self.cut:
                A = synth.tensor(kind, 0, sd)
                xs = [synth.vector("u64", 1, synth.stream_x(k), sd[k]) for k in range(len(sd))]
                self.items.append((A, sd, xs, es))
        self.desc = ("oracle TVC along every mode of " + ", ".join("x".join(map(str, c)) for c in self.cut) +
                     " (the first slabs of each sweep tensor), FP64 and FP32 storage")

    def run_once(self):
        nbytes, secs = 0, 0.0
        for A, sd, xs, es in self.items:
            for k in range(len(sd)):
                t0 = time.perf_counter()
                self.oracle.tvc(A, k, xs[k])
                secs += time.perf_counter() - t0
                nbytes += tvc_bytes(sd, k, es, es)
        return nbytes, secs

    def timed(self, min_seconds):
        nbytes, secs = 0, 0.0
        while secs < min_seconds:
            b, t = self.run_once()
            nbytes += b
            secs += t
        return nbytes / secs / 1e9, secs


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _gbs(nbytes, secs):
    return round(nbytes / secs / 1e9, 2)


def oracle_config_timings(dev, threads):
    """The oracle on each workload at `threads` threads, bounded: the
    128^3 FP64 contraction along every mode and 20 HOPM sweeps (whole); one
    sweep of the oracle's three-buffer HOPM (Algorithm 1) on the first 4
    slabs of the planted 256^4 tensor and on the first 16 slabs of the
    2048^3 tensor stored BF16 and E4M3 (quantised by the oracle); GB/s of
    algorithmic bytes.  Inputs of the large workloads come from the device
    generator (the host generator's bits)."""
    import numpy as np
    import torch
    import oracle
    import synth
    import synth.device as sd
    prev = oracle.set_threads(threads)
    out = {}
    try:
        dims = (128, 128, 128)
        A = synth.tensor("u64", 0, dims)
        t0 = time.perf_counter()
        nb = 0
        for k in range(3):
            oracle.tvc(A, k, synth.vector("u64", 1, synth.stream_x(k), 128))
            nb += tvc_bytes(dims, k, 8, 8)
        out["c1_tvc_GB/s"] = _gbs(nb, time.perf_counter() - t0)
        ones = [np.ones(n) / math.sqrt(n) for n in dims]
        t0 = time.perf_counter()
        oracle.hopm(A, ones, 20)
        sec = time.perf_counter() - t0
        out["c1_hopm20_s"] = round(sec, 3)
        # planted 4 x 256^3 slab sample, one sweep (FP32 storage)
        pd = (4, 256, 256, 256)
        us = [synth.unit_gaussian(0, synth.stream_u(j), 256) for j in range(4)]
        t = torch.empty(math.prod(pd), dtype=torch.float32, device=dev)
        sd.fill(t, "planted", 0, 0, dims=(256,) * 4, us=us)
        Ah = t.cpu().numpy().reshape(pd)
        del t
        t0 = time.perf_counter()
        oracle.hopm3(Ah, [np.ones(n) / math.sqrt(n) for n in pd], 1)
        out["c3_sweep_GB/s"] = _gbs(hopm_bytes(pd, 4, 4), time.perf_counter() - t0)
        del Ah
        # mixed-precision 16 x 2048^2 slab sample, one sweep per format
        md = (16, 2048, 2048)
        t = torch.empty(math.prod(md), dtype=torch.float32, device=dev)
        sd.fill(t, "lognormal", 0, synth.STREAM_A)
        src = t.cpu().numpy().reshape(md)
        del t
        for name, fmt, es in (("bf16", oracle.BF16, 2), ("e4m3", oracle.E4M3, 1)):
            codes, scales = oracle.quantise(src, fmt)
            t0 = time.perf_counter()
            oracle.hopm3(codes, [np.ones(n) / math.sqrt(n) for n in md], 1, scales=scales)
            out[f"c4_{name}_sweep_GB/s"] = _gbs(hopm_bytes(md, es, 4), time.perf_counter() - t0)
    finally:
        oracle.set_threads(prev)
    return out


def cpu_baseline_leg(dev, cores, sampled=None):
    """Timings of the oracle on the host cores (all of them, and one thread),
    and, for `sampled` = [(kind, dims, mode, x, picks)] of timed GPU calls,
    the oracle's values there (plain FP64 sum and the exactly rounded sum)
    with sum_j |a_j x_j|."""
    import oracle
    smp = OracleSample()
    gbs, secs = smp.timed(10.0)
    prev = oracle.set_threads(1)
    try:
        b1, s1 = smp.run_once()
    finally:
        oracle.set_threads(prev)
    res = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": smp.desc,
           "seconds": round(secs, 2),
           "one_thread": {"value": _gbs(b1, s1), "cores": 1, "seconds": round(s1, 2)},
           "configs": {"cores_%d" % cores: oracle_config_timings(dev, cores),
                       "cores_1": oracle_config_timings(dev, 1)}}
    refs = None
    if sampled is not None:
        refs = [sampled_reference(*item) for item in sampled]
    return res, refs


def sampled_reference(kind, dims, mode, x, picks):
    """Oracle values (plain and exactly rounded) and sum |a x| at flat output
    indices `picks` of A x_mode x, from host-generated elements."""
    import numpy as np
    import oracle
    import synth
    nk = dims[mode]
    v = math.prod(dims[mode + 1:])
    j = np.arange(nk, dtype=np.int64)
    plain, exact, mag = (np.empty(len(picks)) for _ in range(3))
    gen = synth.uniform_f64 if kind == "u64" else synth.uniform_f32
    for t, o in enumerate(picks):
        i, l = divmod(int(o), v)
        a = gen(0, synth.STREAM_A, ((i * nk + j) * v + l).astype(np.uint64))
        plain[t] = oracle.tvc(a, 0, x)
        exact[t] = oracle.tvc_exact(a, 0, x)
        mag[t] = np.sum(np.abs(a.astype(np.float64) * x))
    return plain, exact, mag


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    smp = OracleSample()
    for _ in range(args.warmup):
        smp.run_once()
    vals = []
    t1 = time.perf_counter()
    for _ in range(args.steps):
        b, t = smp.run_once()
        vals.append(b / t / 1e9)
    step_s = (time.perf_counter() - t1) / max(1, args.steps)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": smp.desc},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": smp.desc},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ secondary

def _timed(fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# Table 1's FP64 tensors (about 7.5 GB each), every mode: obliviousness to
# order, mode and sizes that are not multiples of 8.
PAPER_SHAPES = [(30623, 30623), (979,) * 3, (175,) * 4, (63,) * 5, (31,) * 6, (19,) * 7, (13,) * 8, (10,) * 9,
                (8,) * 10]


class LoopedCublas:
    """The paper's looped TVC on the GPU (Section 3): one GEMV for the last
    mode, otherwise u equally sized vector-matrix products in one
    cublasDgemvStridedBatched call.  A comparator for the bench only (loaded
    from the CUDA toolkit's cuBLAS through ctypes), never a library path."""

    def __init__(self, stream_ptr):
        import ctypes
        lib = None
        for name in ("libcublas.so.13", "libcublas.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise OSError("cuBLAS not found")
        self.ct = ctypes
        self.lib = lib
        self.h = ctypes.c_void_p()
        if lib.cublasCreate_v2(ctypes.byref(self.h)) != 0:
            raise OSError("cublasCreate failed")
        lib.cublasSetStream_v2(self.h, ctypes.c_void_p(stream_ptr))
        P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        lib.cublasDgemv_v2.argtypes = [P, I, I, I, P, P, I, P, I, P, P, I]
        lib.cublasDgemvStridedBatched.argtypes = [P, I, I, I, P, P, I, L, P, I, L, P, P, I, L, I]
        self.one = ctypes.c_double(1.0)
        self.zero = ctypes.c_double(0.0)

    def tvc(self, A, dims, k, x, y):
        ct = self.ct
        u = math.prod(dims[:k])
        nk = dims[k]
        v = math.prod(dims[k + 1:])
        a, xp, yp = ct.c_void_p(A.data_ptr()), ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr())
        if v == 1:  # Y = A^{u x n_k} x: the row-major matrix is n_k x u column-major, transposed
            rc = self.lib.cublasDgemv_v2(self.h, 1, nk, u, ct.byref(self.one), a, nk, xp, 1, ct.byref(self.zero),
                                         yp, 1)
        else:  # u products x^T A_i^{n_k x v}: A_i is v x n_k column-major
            rc = self.lib.cublasDgemvStridedBatched(self.h, 0, v, nk, ct.byref(self.one), a, v, nk * v, xp, 1, 0,
                                                    ct.byref(self.zero), yp, 1, v, u)
        if rc != 0:
            raise RuntimeError(f"cuBLAS status {rc}")

    def close(self):
        self.lib.cublasDestroy_v2(self.h)


def paper_shapes(dev, peak, index=0):
    """Per-mode GB/s of the native TVC and of the looped cuBLAS TVC on
    Table 1's FP64 tensors; mean and sample std over all modes; SM clocks
    sampled during the whole measurement."""
    import torch
    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg
    try:
        looped = LoopedCublas(torch.cuda.current_stream().cuda_stream)
    except OSError as e:
        looped = None
        why = str(e)
    native, loop, worst = {}, {}, 0.0
    sampler = ClockSampler(index)
    sampler.start()
    for dims in PAPER_SHAPES:
        N = math.prod(dims)
        A = torch.empty(N, dtype=torch.float64, device=dev)
        sd.fill(A, "u64", 0, synth.STREAM_A)
        for k in range(len(dims)):
            x = torch.from_numpy(synth.vector("u64", 1, synth.stream_x(k), dims[k])).to(dev)
            y = torch.empty(N // dims[k], dtype=torch.float64, device=dev)
            nb = tvc_bytes(dims, k, 8, 8)
            name = f"{dims[0]}^{len(dims)}:k{k}"
            ms = _timed(lambda: tg.tvc(A, k, x, y=y, shape=dims), 5, warm=2)
            native[name] = nb / (ms / 1e3) / 1e9
            if looped is not None:
                y2 = torch.empty_like(y)
                ms2 = _timed(lambda: looped.tvc(A, dims, k, x, y2), 5, warm=2)
                loop[name] = nb / (ms2 / 1e3) / 1e9
                worst = max(worst, float(((y2 - y).abs().max() / y.abs().max().clamp_min(1e-300)).item()))
                del y2
            del x, y
        del A
        torch.cuda.empty_cache()

    def summary(d):
        vals = list(d.values())
        return {"mean_GBs": statistics.mean(vals), "std_GBs": statistics.stdev(vals),
                "mean_frac": statistics.mean(vals) / peak, "std_frac": statistics.stdev(vals) / peak,
                "min_frac": min(vals) / peak, "max_frac": max(vals) / peak}

    clocks = sampler.stop()
    out = {"shapes": "Table 1 FP64 tensors 30623^2, 979^3, 175^4, 63^5, 31^6, 19^7, 13^8, 10^9, 8^10; every mode",
           "clocks": clocks,
           "native": summary(native), "native_per_mode_GBs": {n: round(v, 1) for n, v in native.items()}}
    if looped is not None:
        out["looped_cublas"] = summary(loop)
        out["looped_cublas_per_mode_GBs"] = {n: round(v, 1) for n, v in loop.items()}
        out["looped_vs_native_max_rel_diff"] = worst
        looped.close()
    else:
        out["looped_cublas"] = {"unavailable": why}
    return out


def hopm_bytes(dims, es, vs):
    """Algorithmic bytes of one sweep of the two-pass HOPM: A read twice,
    W_1 and later prefix tensors written and read once, T written and read."""
    N = math.prod(dims)
    d = len(dims)
    b = 2 * N * es
    b += 2 * (N // dims[1]) * vs  # T = A x_1 x_1
    w = N // dims[0]
    for j in range(1, d):
        b += 2 * w * vs  # W_j written, then read
        if j + 1 < d:
            w //= dims[j]
    return b


def golden_hopm():
    """The FP64 oracle's results for the full-size power-method workloads,
    stored by tests/golden/make_fullsize_hopm.py (oracle only), or None."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "hopm_fullsize.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def _rel(a, b):
    return abs(a - b) / abs(b)


def hopm_workloads(dev):
    """The two full-size power-method workloads, timed, with their error
    against the FP64 oracle's stored results:
    planted rank-1 + noise 256^4 FP32 (50 sweeps, tol 1e-8, from a start
    overlapping the planted factors), and 2048^3 N(0,1)exp(U[-3,3]) stored
    FP32, BF16 and E4M3 with per-slab scales (30 sweeps from all-ones).
    Returns (summary for the result line, details)."""
    import numpy as np
    import torch
    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg
    gold = golden_hopm()
    summary, detail = {}, {}
    # planted rank-1 + noise
    dims = (256, 256, 256, 256)
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    A = torch.empty(math.prod(dims), dtype=torch.float32, device=dev)
    sd.fill(A, "planted", 0, 0, dims=dims, us=us)
    ws = torch.empty(tg.hopm_workspace_size(dims, tg.F32), dtype=torch.uint8, device=dev)
    pert = []
    for j, n in enumerate(dims):
        v = us[j] + synth.unit_gaussian(1, synth.stream_u(j), n)
        pert.append(torch.from_numpy((v / np.linalg.norm(v)).astype(np.float32)).to(dev))
    r = tg.hopm(A, pert, 50, 1e-8, shape=dims, workspace=ws)
    torch.cuda.synchronize()
    sub = max(math.sqrt(max(0.0, 1 - float(np.dot(x.cpu().numpy().astype(np.float64), u)) ** 2))
              for x, u in zip(r.x, us))
    ms = _timed(lambda: tg.hopm(A, pert, 50, 0.0, shape=dims, workspace=ws), 2)
    c3 = {"lambda": round(r.lam.item(), 6), "sweeps": int(r.sweeps.item()), "subspace_err": round(sub, 5),
          "sweeps_per_s": round(50 / (ms / 1e3), 1),
          "GB/s": round(50 * hopm_bytes(dims, 4, 4) / (ms / 1e3) / 1e9, 1)}
    if gold and "planted" in gold:
        c3["lambda_rel_err_vs_oracle"] = float("%.3g" % _rel(r.lam.item(), gold["planted"]["lam"]))
    summary["hopm_c3"] = c3
    ones = [torch.full((n,), 1 / math.sqrt(n), dtype=torch.float32, device=dev) for n in dims]
    rr = tg.hopm(A, ones, 50, 1e-8, shape=dims, workspace=ws)
    torch.cuda.synchronize()
    detail["hopm_planted_from_ones"] = {"lambda": rr.lam.item(), "sweeps": int(rr.sweeps.item())}
    del A, ws, r, rr
    torch.cuda.empty_cache()
    # 2048^3 stored FP32 / BF16 / E4M3
    dims = (2048, 2048, 2048)
    src = torch.empty(math.prod(dims), dtype=torch.float32, device=dev)
    sd.fill(src, "lognormal", 0, synth.STREAM_A)
    xs0 = [torch.full((n,), 1 / math.sqrt(n), dtype=torch.float32, device=dev) for n in dims]
    res = {}
    gm = gold.get("mixed") if gold else None
    for name, code in (("f32", tg.F32), ("bf16", tg.BF16), ("e4m3", tg.E4M3)):
        if code == tg.F32:
            A, sc = src, None
        else:
            A, sc, _ = tg.quantise(src.view(dims), code)
            A = A.view(-1)
        ws = torch.empty(tg.hopm_workspace_size(dims, code), dtype=torch.uint8, device=dev)
        r = tg.hopm(A, xs0, 30, 0.0, scales=sc, shape=dims, workspace=ws)
        torch.cuda.synchronize()
        lam = r.lam.item()
        ms = _timed(lambda: tg.hopm(A, xs0, 30, 0.0, scales=sc, shape=dims, workspace=ws), 2)
        es = {"f32": 4, "bf16": 2, "e4m3": 1}[name]
        e = {"sweeps_per_s": round(30 / (ms / 1e3), 1),
             "GB/s": round(30 * hopm_bytes(dims, es, 4) / (ms / 1e3) / 1e9, 1), "lambda": round(lam, 6)}
        if gm:
            # against the oracle on the binary32 source (storage + kernel error)
            e["lambda_rel_err_vs_oracle"] = float("%.3g" % _rel(lam, gm["f32"]["lam"]))
            if name != "f32":  # against the oracle on the same stored codes (kernel error)
                e["kernel_rel_err"] = float("%.3g" % _rel(lam, gm[name]["lam"]))
        res[name] = e
        del A, ws, r
        torch.cuda.empty_cache()
    res["bf16_over_f32_sweeps"] = round(res["bf16"]["sweeps_per_s"] / res["f32"]["sweeps_per_s"], 3)
    res["e4m3_over_f32_sweeps"] = round(res["e4m3"]["sweeps_per_s"] / res["f32"]["sweeps_per_s"], 3)
    summary["hopm_c4"] = res
    del src
    torch.cuda.empty_cache()
    return summary, detail


def secondary(dev):
    """HOPM 128^3, batched, TMC and MTTKRP figures (details, not part of `value`)."""
    import numpy as np
    import torch
    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg
    out = {}
    # 128^3 FP64, 20 sweeps from normalised ones
    dims = (128, 128, 128)
    A = torch.empty(math.prod(dims), dtype=torch.float64, device=dev)
    sd.fill(A, "u64", 0, synth.STREAM_A)
    xs = [torch.full((n,), 1 / math.sqrt(n), dtype=torch.float64, device=dev) for n in dims]
    ws = torch.empty(tg.hopm_workspace_size(dims, tg.F64), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: tg.hopm(A, xs, 20, shape=dims, workspace=ws), 5)
    # the same 20 sweeps replayed from a CUDA graph (no launch overhead)
    xg = [v.clone() for v in xs]
    hopm_graph = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        tg.hopm(A, xg, 20, shape=dims, workspace=ws, inplace=True, stream=gs)  # warm-up outside capture
        with torch.cuda.graph(hopm_graph, stream=gs):
            tg.hopm(A, xg, 20, shape=dims, workspace=ws, inplace=True, stream=gs)
    torch.cuda.current_stream().wait_stream(gs)
    gms = _timed(hopm_graph.replay, 10)
    out["hopm_128cube_f64_20sweeps"] = {"ms": ms, "sweeps_per_s": 20 / (ms / 1e3),
                                        "graph_ms": gms, "graph_sweeps_per_s": 20 / (gms / 1e3),
                                        "GB/s_effective_L2": 20 * hopm_bytes(dims, 8, 8) / (gms / 1e3) / 1e9,
                                        "note": "16.8 MB tensor: L2-resident"}
    del A, ws
    torch.cuda.empty_cache()
    # batched: 4096 FP32 tensors (order 3/4, dims U[8,192], <= 2^24 elements)
    spec = batched_spec(4096)
    total = sum(math.prod(dd) for dd, _ in spec)
    pool = torch.empty(total, dtype=torch.float32, device=dev)
    sd.fill(pool, "u32", 0, synth.STREAM_A)
    gApool = torch.empty(total, dtype=torch.float32, device=dev)
    items, hitems, off, nbytes = [], [], 0, 0
    for b, (dd, mode) in enumerate(spec):
        N = math.prod(dd)
        A = pool[off:off + N]
        gA = gApool[off:off + N]
        off += N
        x = torch.full((dd[mode],), 0.5, dtype=torch.float32, device=dev)
        gy = torch.full((N // dd[mode],), 0.25, dtype=torch.float32, device=dev)
        items.append(dict(A=A, shape=dd, mode=mode, x=x, y=torch.empty_like(gy), gy=gy,
                          gx=torch.empty(dd[mode], dtype=torch.float32, device=dev), gA=gA))
        nbytes += 2 * N * 4 + N * 4 + 2 * (N // dd[mode]) * 4 + N * 4  # A twice, gy, y, gA write
        hitems.append(dict(A=A, shape=dd, x=[torch.full((n,), 1 / math.sqrt(n), dtype=torch.float32, device=dev)
                                             for n in dd]))
    batch = tg.TVCBatch(items)
    batch.run()
    ms = _timed(batch.run, 3)
    hb = tg.HOPMBatch(hitems, 10)
    hb.run()
    hms = _timed(hb.run, 2)
    hbytes = sum(10 * hopm_bytes(dd, 4, 4) for dd, _ in spec)
    out["batched_4096"] = {"elements": total, "fwd_bwd_ms": ms, "fwd_bwd_GB/s": nbytes / (ms / 1e3) / 1e9,
                           "hopm10_ms": hms, "hopm10_GB/s": hbytes / (hms / 1e3) / 1e9,
                           "note": "one persistent launch each; effective GB/s (part of the data is L2-resident)"}
    del pool, gApool, items, hitems, batch, hb
    torch.cuda.empty_cache()
    # tensor-matrix contraction (Section 1's TMC, the HOOI / CP-ALS building
    # block): 1024^3 FP32, R = 4 and 8 rows of X, every mode; algorithmic bytes
    dims = (1024, 1024, 1024)
    N = math.prod(dims)
    A = torch.empty(N, dtype=torch.float32, device=dev)
    sd.fill(A, "u32", 0, synth.STREAM_A)
    res = {}
    for R in (4, 8):
        for k in range(3):
            X = torch.from_numpy(synth.tensor("u32", 1, (R, dims[k]), synth.stream_x(k))).to(dev)
            Y = torch.empty(N // dims[k] * R, dtype=torch.float32, device=dev)
            ws = torch.empty(max(1, tg.tmc_workspace_size(dims, k, R, tg.F32)), dtype=torch.uint8, device=dev)
            ms = _timed(lambda: tg.tmc(A, k, X, Y=Y, shape=dims, workspace=ws), 5)
            res[f"R{R}_mode{k}_GB/s"] = (N * 4 + X.numel() * 4 + Y.numel() * 4) / (ms / 1e3) / 1e9
            del X, Y, ws
    out["tmc_1024^3_f32"] = res
    # MTTKRP (CP-ALS building block) on the same tensor: R = 8 factor columns, every mode
    res = {}
    for k in range(3):
        facs = [None if m == k else torch.from_numpy(synth.tensor("u32", 1, (n, 8), 20 + m)).to(dev)
                for m, n in enumerate(dims)]
        ws = torch.empty(max(1, tg.mttkrp_workspace_size(dims, k, 8, tg.F32)), dtype=torch.uint8, device=dev)
        ms = _timed(lambda: tg.mttkrp(A, k, facs, workspace=ws, shape=dims), 5)
        nbytes = N * 4 + sum(f.numel() * 4 for f in facs if f is not None) + dims[k] * 8 * 4
        res[f"R8_mode{k}_GB/s"] = nbytes / (ms / 1e3) / 1e9
        del facs, ws
    out["mttkrp_1024^3_f32"] = res
    del A
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------- single cases (profiling)

def batched_spec(count, seed=0):
    """The batched workload's tensors: order 3 or 4 (seeded coin), dims
    U[8,192], redrawn above 2^24 elements, a random contraction mode."""
    import numpy as np
    rng = np.random.default_rng(seed)
    spec = []
    for _ in range(count):
        d = 3 if rng.random() < 0.5 else 4
        while True:
            dd = tuple(int(n) for n in rng.integers(8, 193, size=d))
            if math.prod(dd) <= (1 << 24):
                break
        spec.append((dd, int(rng.integers(0, d))))
    return spec


def run_case(argv):
    """One contraction case, repeated, for profiling (ncu) and quick timing:

        python bench.py --case tvc --dims 512 1024 1024 --mode 1 --dtype f64 --reps 3
        python bench.py --case tvc --dims 1024 1024 1024 --mode 0 --dtype f32 --tmc 4
        python bench.py --case batched --count 128 --what tvc --reps 3

    tvc: fills A (uniform [-1, 1), seed 0) on the device, runs `reps`
    contractions (--tmc R: the tensor-matrix contraction with an R-row
    matrix; --mttkrp R: the MTTKRP with R-column factors) and prints the
    CUDA-event time and the GB/s of the last one.  batched: the batched
    workload at --count tensors; --what tvc (forward), fwdbwd (forward + gx
    + rank-1 gA), gx, ga (one adjoint), hopm (10 sweeps per tensor)."""
    import torch
    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg

    ap = argparse.ArgumentParser(prog="bench.py --case")
    ap.add_argument("case", choices=["tvc", "batched"])
    ap.add_argument("--dims", type=int, nargs="+")
    ap.add_argument("--mode", type=int, default=0)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16", "e4m3", "f16", "f32d"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tmc", type=int, default=0, help="rows of X (tensor-matrix contraction); 0: TVC")
    ap.add_argument("--mttkrp", type=int, default=0, help="columns of the factor matrices (MTTKRP); 0: TVC")
    ap.add_argument("--count", type=int, default=128)
    ap.add_argument("--what", default="tvc", choices=["tvc", "fwdbwd", "gx", "ga", "hopm"])
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_last(fn):
        ms = 0.0
        for _ in range(a.reps):
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        return ms, out

    if a.case == "batched":
        spec = batched_spec(a.count)
        total = sum(math.prod(dd) for dd, _ in spec)
        pool = torch.empty(total, dtype=torch.float32, device=dev)
        sd.fill(pool, "u32", 0, synth.STREAM_A)
        items, off, nbytes = [], 0, 0
        f32 = dict(dtype=torch.float32, device=dev)
        for dd, mode in spec:
            N = math.prod(dd)
            A = pool[off:off + N]
            off += N
            if a.what == "hopm":
                items.append(dict(A=A, shape=dd, x=[torch.full((n,), 1 / math.sqrt(n), **f32) for n in dd]))
                nbytes += 10 * (2 * N * 4)
                continue
            x = torch.full((dd[mode],), 0.5, **f32)
            gy = torch.full((N // dd[mode],), 0.25, **f32)
            it = dict(A=A, shape=dd, mode=mode, x=x)
            nbytes += N * 4 + (N // dd[mode]) * 4
            if a.what == "gx":
                it.update(gy=gy, gx=torch.empty(dd[mode], **f32))
            elif a.what == "ga":
                it.update(gy=gy, gA=torch.empty(N, **f32))
            else:
                it.update(y=torch.empty(N // dd[mode], **f32))
                if a.what == "fwdbwd":
                    it.update(gy=gy, gx=torch.empty(dd[mode], **f32), gA=torch.empty(N, **f32))
                    nbytes += N * 4 + (N // dd[mode]) * 4 + N * 4
            items.append(it)
        batch = tg.HOPMBatch(items, 10) if a.what == "hopm" else tg.TVCBatch(items)
        ms, _ = timed_last(batch.run)
        print(f"{a.count} tensors ({total / 1e9:.2f}e9 elements) {a.what}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")
        return 0

    if not a.dims:
        ap.error("--dims is required for --case tvc")
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    kind = "u64" if a.dtype == "f64" else "u32"
    N = math.prod(a.dims)
    A = torch.empty(N, dtype=dt, device=dev)
    sd.fill(A, kind, 0, synth.STREAM_A)
    scales = None
    if a.dtype in ("bf16", "e4m3", "f16"):
        A, scales, _ = tg.quantise(A.view(a.dims), {"bf16": tg.BF16, "e4m3": tg.E4M3, "f16": tg.F16}[a.dtype])
        A = A.view(-1)
    xkind = "u64" if a.dtype == "f32d" else kind  # single-double: FP32 storage, FP64 vectors
    code = tg.F32D if a.dtype == "f32d" else tg.dtype_code(A)
    nk = a.dims[a.mode]
    if a.mttkrp:
        R = a.mttkrp
        facs = [None if m == a.mode else torch.from_numpy(synth.tensor(xkind, 1, (n, R), 20 + m)).to(dev)
                for m, n in enumerate(a.dims)]
        ws = torch.empty(max(1, tg.mttkrp_workspace_size(a.dims, a.mode, R, code)), dtype=torch.uint8, device=dev)
        ms, M = timed_last(lambda: tg.mttkrp(A, a.mode, facs, scales=scales, workspace=ws, shape=a.dims))
        nbytes = N * A.element_size() + sum(f.numel() * f.element_size() for f in facs if f is not None) \
            + M.numel() * M.element_size()
        print(f"dims={a.dims} mode={a.mode} {a.dtype} mttkrp R={R}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")
        return 0
    R = max(1, a.tmc)
    if a.tmc:
        x = torch.from_numpy(synth.tensor(xkind, 1, (R, nk), synth.stream_x(a.mode))).to(dev)
        y = torch.empty(N // nk * R, dtype=x.dtype, device=dev)
        ws = torch.empty(max(1, tg.tmc_workspace_size(a.dims, a.mode, R, code)), dtype=torch.uint8, device=dev)
        fn = lambda: tg.tmc(A, a.mode, x, Y=y, shape=a.dims, scales=scales, workspace=ws)  # noqa: E731
    else:
        x = torch.from_numpy(synth.vector(xkind, 1, synth.stream_x(a.mode), nk)).to(dev)
        y = torch.empty(N // nk, dtype=x.dtype, device=dev)
        ws = torch.empty(max(1, tg.tvc_workspace_size(a.dims, a.mode, code)), dtype=torch.uint8, device=dev)
        fn = lambda: tg.tvc(A, a.mode, x, y=y, shape=a.dims, scales=scales, workspace=ws)  # noqa: E731
    ms, _ = timed_last(fn)
    nbytes = N * A.element_size() + x.numel() * x.element_size() + y.numel() * y.element_size()
    what = f"tmc R={R}" if a.tmc else "tvc"
    print(f"dims={a.dims} mode={a.mode} {a.dtype} {what}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")
    return 0


# ------------------------------------------------------------------- main

def main(argv=None):
    argv = sys.argv[1:] if argv is None else list(argv)
    # Tensors through torch's expandable segments (physical memory mapped in
    # 2 MB granules): after the workloads' earlier allocations and frees, a
    # fresh multi-GB tensor could otherwise be backed by small pages, and a
    # contraction that walks every row of the whole tensor at once (mode 0
    # of 979^3: 979 rows 7.6 MB apart in flight) lost 30% of its bandwidth
    # to address-translation misses (4410 against 6290 GB/s).  Takes effect
    # only when set before torch's first CUDA allocation; a setting of the
    # caller's own (under either name) is kept.
    # (The older variable name: torch 2.9 warns that it is deprecated but
    # measured to apply it, while the newer PYTORCH_ALLOC_CONF left that mode
    # at 4545 GB/s.)
    if "PYTORCH_ALLOC_CONF" not in os.environ and "PYTORCH_CUDA_ALLOC_CONF" not in os.environ:
        os.environ["PYTORCH_CUDA_ALLOC_CONF"] = "expandable_segments:True"
    if argv and argv[0] == "--case":
        return run_case(argv[1:])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--detail", action="store_true", help="per-mode table on stderr")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the HOPM / batched figures")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    stream = torch.cuda.current_stream()
    # Inputs, resident in HBM.
    calls = []
    tensors = []
    for code, dt, kind in ((tg.F64, torch.float64, "u64"), (tg.F32, torch.float32, "u32")):
        es = 8 if code == tg.F64 else 4
        for dims in TENSORS:
            N = math.prod(dims)
            A = torch.empty(N, dtype=dt, device=dev)
            sd.fill(A, kind, 0, synth.STREAM_A)
            tensors.append((A, dims, code))
            for k in range(len(dims)):
                xh = synth.vector(kind, 1, synth.stream_x(k), dims[k])
                x = torch.from_numpy(xh).to(dev)
                y = torch.empty(N // dims[k], dtype=dt, device=dev)
                calls.append(dict(A=A, dims=dims, k=k, x=x, xh=xh, y=y, code=code,
                                  bytes=tvc_bytes(dims, k, es, es), name=f"{'f64' if code == tg.F64 else 'f32'}:"
                                  f"{'x'.join(map(str, dims))}:k{k}", v=math.prod(dims[k + 1:])))
    torch.cuda.synchronize()
    step_bytes = sum(c["bytes"] for c in calls)

    def step(evs=None):
        for ci, c in enumerate(calls):
            if evs is not None:
                evs[ci][0].record(stream)
            tg.tvc(c["A"], c["k"], c["x"], y=c["y"], shape=c["dims"])
            if evs is not None:
                evs[ci][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = tg.kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = tg.kernel_launches() - launches0
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms = max_over_ranks(elapsed_ms, pg, dev)
    per_call = [statistics.mean(evs[s][ci][0].elapsed_time(evs[s][ci][1]) for s in range(args.steps))
                for ci in range(len(calls))]
    value = world * step_bytes * args.steps / (elapsed_ms / 1e3) / 1e9

    # Dominant kernel: the FP64 column kernel (modes with v >= 32), which
    # carries most of the step's time.
    peak, peak_kind = peaks()
    dom = [ci for ci, c in enumerate(calls) if c["code"] == tg.F64 and c["v"] >= 32]
    dom_bytes = sum(calls[ci]["bytes"] for ci in dom)
    dom_ms = sum(per_call[ci] for ci in dom)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    rec = traffic_record()
    avg_dom_bytes = dom_bytes / max(1, len(dom))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind, "kernel": "tvc_cols_kernel<F64> (FP64 contraction, v >= 32)",
                "launches_timed": len(dom) * args.steps, "algorithmic_bytes_per_launch": avg_dom_bytes,
                "traffic": (rec["traffic_over_algorithmic"] * avg_dom_bytes if rec else None),
                "traffic_note": ("ncu dram read+write of a 512x1024x1024 capture, scaled per launch by the "
                                 "elements processed" if rec else "no capture of the current kernel source")}
    f64_ms = sum(per_call[ci] for ci, c in enumerate(calls) if c["code"] == tg.F64)
    f64_bytes = sum(c["bytes"] for c in calls if c["code"] == tg.F64)
    f32_ms = sum(per_call[ci] for ci, c in enumerate(calls) if c["code"] == tg.F32)
    f32_bytes = sum(c["bytes"] for c in calls if c["code"] == tg.F32)
    per_mode = {c["name"]: round(c["bytes"] / (per_call[ci] / 1e3) / 1e9, 1) for ci, c in enumerate(calls)}
    if args.detail and rank == 0:
        for name, gbs in per_mode.items():
            print(f"{name:40s} {gbs:8.1f} GB/s  {100 * gbs / peak:5.1f}%", file=sys.stderr)

    # Outputs of the timed calls at sampled indices (checked against the
    # oracle in the CPU-baseline leg below).
    rng = np.random.default_rng(0)
    sampled, got_sampled = [], []
    for c in calls:
        uv = c["y"].numel()
        picks = np.unique(np.concatenate([rng.integers(0, uv, size=32, dtype=np.int64), [0, uv - 1]]))
        got_sampled.append(c["y"].reshape(-1)[torch.from_numpy(picks).to(dev)].double().cpu().numpy())
        sampled.append(("u64" if c["code"] == tg.F64 else "u32", c["dims"], c["k"], c["xh"], picks))

    # End to end through the public API: inputs from pinned host memory,
    # results read back, every step.
    e2e = None
    if not args.no_e2e:
        hostA = []
        for A, dims, code in tensors:
            h = torch.empty(A.numel(), dtype=A.dtype, pin_memory=True)
            h.copy_(A)
            hostA.append(h)
        hostY = [torch.empty(c["y"].numel(), dtype=c["y"].dtype, pin_memory=True) for c in calls]
        hostX = [c["x"].cpu().pin_memory() for c in calls]
        h2d = sum(h.numel() * h.element_size() for h in hostA) + sum(h.numel() * h.element_size() for h in hostX)
        d2h = sum(h.numel() * h.element_size() for h in hostY)
        torch.cuda.synchronize()

        def e2e_step():
            ci = 0
            for (A, dims, code), h in zip(tensors, hostA):
                A.copy_(h, non_blocking=True)
                for k in range(len(dims)):
                    c = calls[ci]
                    c["x"].copy_(hostX[ci], non_blocking=True)
                    tg.tvc(A, k, c["x"], y=c["y"], shape=dims)
                    hostY[ci].copy_(c["y"], non_blocking=True)
                    ci += 1

        e2e_step()
        torch.cuda.synchronize()
        k2 = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * step_bytes * k2 / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k2}
        del hostA, hostY

    # free the sweep's tensors before the other workloads
    n_calls = len(calls)
    del tensors, calls, evs
    torch.cuda.empty_cache()
    hopm_sum, detail = {}, {}
    if world == 1 and not args.no_secondary:
        hopm_sum, detail = hopm_workloads(dev)
        detail.update(secondary(dev))
        detail["paper_shapes_fp64"] = paper_shapes(dev, peak, local)

    cpu = None
    fp_err = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, refs = cpu_baseline_leg(dev, oracle_threads(), sampled)
        for code_name in ("f64", "f32"):
            sel = [i for i, smp in enumerate(sampled) if (smp[0] == "u64") == (code_name == "f64")]
            got = np.concatenate([got_sampled[i] for i in sel])
            plain = np.concatenate([refs[i][0] for i in sel])
            fp_err[code_name] = {"rel_l2_vs_oracle": float("%.3g" % (np.linalg.norm(got - plain) /
                                                                       np.linalg.norm(plain))),
                                 "outputs_checked": int(got.size)}
            if code_name == "f64":
                exact = np.concatenate([refs[i][1] for i in sel])
                mag = np.concatenate([refs[i][2] for i in sel])
                # the FP64 error model: |y - y_exact| <= c 2^-46 sum|a x| (c = 4 tested)
                fp_err[code_name]["max_err_over_2^-46_sum|ax|"] = float(
                    "%.3g" % np.max(np.abs(got - exact) / (2.0 ** -46 * mag)))

    if rank == 0:
        detail["per_mode_GBs"] = per_mode
        print("detail " + json.dumps(detail), file=sys.stderr, flush=True)
        f64_modes = [v for n, v in per_mode.items() if n.startswith("f64")]
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (float-float products) + f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "tvcs_per_step": n_calls, "bytes_per_step": step_bytes,
                       "l2": "inputs larger than L2 (smallest tensor 1.07 GB); no flush needed",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "frac_of_peak": round(value / world / peak, 4),
            "fp64": dict({"GB/s": round(f64_bytes / (f64_ms / 1e3) / 1e9, 1),
                          "frac": round(f64_bytes / (f64_ms / 1e3) / 1e9 / peak, 4),
                          "min_mode_frac": round(min(f64_modes) / peak, 4),
                          "mean_mode_frac": round(statistics.mean(f64_modes) / peak, 4),
                          "std_mode_frac": round(statistics.stdev(f64_modes) / peak, 4)}, **fp_err.get("f64", {})),
            "fp32": dict({"GB/s": round(f32_bytes / (f32_ms / 1e3) / 1e9, 1),
                          "frac": round(f32_bytes / (f32_ms / 1e3) / 1e9 / peak, 4)}, **fp_err.get("f32", {})),
        }
        line.update(hopm_sum)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
