"""The batched workload (FP32 tensors of order 3 or 4, dims U[8,192], at
most 2^24 elements each, a random contraction mode; seeded), at a chosen
tensor count, repeated, for profiling (ncu) and quick timing.

    python -m paper_2501_03121_gb300.profile_batched --count 128 --what tvc --reps 3

--what tvc: forward contraction only; fwdbwd: forward + gx + rank-1 gA;
gx, ga: one adjoint alone; hopm: 10 power-method sweeps per tensor.  Prints the time of the last run
and the effective GB/s (algorithmic bytes / time).
"""
import argparse
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def spec_of(count, seed=0):
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


def main(argv=None):
    import torch

    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=128)
    ap.add_argument("--what", default="tvc", choices=["tvc", "fwdbwd", "gx", "ga", "hopm"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    spec = spec_of(a.count)
    total = sum(math.prod(dd) for dd, _ in spec)
    pool = torch.empty(total, dtype=torch.float32, device=dev)
    sd.fill(pool, "u32", 0, synth.STREAM_A)
    items, off, nbytes = [], 0, 0
    for dd, mode in spec:
        N = math.prod(dd)
        A = pool[off:off + N]
        off += N
        if a.what == "hopm":
            items.append(dict(A=A, shape=dd, x=[torch.full((n,), 1 / math.sqrt(n), dtype=torch.float32,
                                                            device=dev) for n in dd]))
            nbytes += 10 * (2 * N * 4)
            continue
        x = torch.full((dd[mode],), 0.5, dtype=torch.float32, device=dev)
        gy = torch.full((N // dd[mode],), 0.25, dtype=torch.float32, device=dev)
        if a.what == "gx":
            items.append(dict(A=A, shape=dd, mode=mode, x=x, gy=gy, gx=torch.empty(dd[mode], dtype=torch.float32,
                                                                                  device=dev)))
            nbytes += N * 4 + (N // dd[mode]) * 4
            continue
        if a.what == "ga":
            items.append(dict(A=A, shape=dd, mode=mode, x=x, gy=gy, gA=torch.empty(N, dtype=torch.float32, device=dev)))
            nbytes += N * 4 + (N // dd[mode]) * 4
            continue
        it = dict(A=A, shape=dd, mode=mode, x=x, y=torch.empty(N // dd[mode], dtype=torch.float32, device=dev))
        nbytes += N * 4 + (N // dd[mode]) * 4
        if a.what == "fwdbwd":
            it.update(gy=torch.full((N // dd[mode],), 0.25, dtype=torch.float32, device=dev),
                      gx=torch.empty(dd[mode], dtype=torch.float32, device=dev),
                      gA=torch.empty(N, dtype=torch.float32, device=dev))
            nbytes += N * 4 + (N // dd[mode]) * 4 + N * 4
        items.append(it)
    batch = tg.HOPMBatch(items, 10) if a.what == "hopm" else tg.TVCBatch(items)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(a.reps):
        e0.record()
        batch.run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    print(f"{a.count} tensors ({total / 1e9:.2f}e9 elements) {a.what}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")


if __name__ == "__main__":
    main()
