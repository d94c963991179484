"""One contraction case, repeated, for profiling (ncu) and quick timing.

    python -m paper_2501_03121_gb300.profile_case --dims 512 1024 1024 --mode 1 --dtype f64 --reps 3

Fills A (uniform [-1, 1), seed 0) on the device, runs `reps` contractions
and prints the CUDA-event time and achieved GB/s of the last one.  With
--tmc R the contraction is the tensor-matrix one with an R-row matrix;
with --mttkrp R it is the MTTKRP with R-column factor matrices.
"""
import argparse
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import synth
    import synth.device as sd
    import paper_2501_03121_gb300 as tg

    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs="+", required=True)
    ap.add_argument("--mode", type=int, default=0)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16", "e4m3", "f16", "f32d"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tmc", type=int, default=0, help="rows of X (tensor-matrix contraction); 0: TVC")
    ap.add_argument("--mttkrp", type=int, default=0, help="columns of the factor matrices (MTTKRP); 0: TVC")
    a = ap.parse_args(argv)
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    kind = "u64" if a.dtype == "f64" else "u32"
    N = math.prod(a.dims)
    A = torch.empty(N, dtype=dt, device="cuda")
    sd.fill(A, kind, 0, synth.STREAM_A)
    scales = None
    if a.dtype in ("bf16", "e4m3", "f16"):
        A, scales, _ = tg.quantise(A.view(a.dims), {"bf16": tg.BF16, "e4m3": tg.E4M3, "f16": tg.F16}[a.dtype])
        A = A.view(-1)
    xkind = "u64" if a.dtype == "f32d" else kind  # single-double: FP32 storage, FP64 vectors
    code = tg.F32D if a.dtype == "f32d" else tg.dtype_code(A)
    R = max(1, a.tmc)
    nk = a.dims[a.mode]
    if a.mttkrp:
        R = a.mttkrp
        facs = [None if m == a.mode else torch.from_numpy(synth.tensor(xkind, 1, (n, R), 20 + m)).cuda()
                for m, n in enumerate(a.dims)]
        ws = torch.empty(max(1, tg.mttkrp_workspace_size(a.dims, a.mode, R, code)), dtype=torch.uint8,
                         device="cuda")
        fn = lambda: tg.mttkrp(A, a.mode, facs, scales=scales, workspace=ws, shape=a.dims)  # noqa: E731
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(a.reps):
            e0.record()
            M = fn()
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nbytes = N * A.element_size() + sum(f.numel() * f.element_size() for f in facs if f is not None) \
            + M.numel() * M.element_size()
        print(f"dims={a.dims} mode={a.mode} {a.dtype} mttkrp R={R}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")
        return
    if a.tmc:
        x = torch.from_numpy(synth.tensor(xkind, 1, (R, nk), synth.stream_x(a.mode))).cuda()
        y = torch.empty(N // nk * R, dtype=x.dtype, device="cuda")
        ws = torch.empty(max(1, tg.tmc_workspace_size(a.dims, a.mode, R, code)), dtype=torch.uint8, device="cuda")
    else:
        x = torch.from_numpy(synth.vector(xkind, 1, synth.stream_x(a.mode), nk)).cuda()
        y = torch.empty(N // nk, dtype=x.dtype, device="cuda")
        ws = torch.empty(max(1, tg.tvc_workspace_size(a.dims, a.mode, code)), dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(a.reps):
        e0.record()
        if a.tmc:
            tg.tmc(A, a.mode, x, Y=y, shape=a.dims, scales=scales, workspace=ws)
        else:
            tg.tvc(A, a.mode, x, y=y, shape=a.dims, scales=scales, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    nbytes = N * A.element_size() + x.numel() * x.element_size() + y.numel() * y.element_size()
    what = f"tmc R={R}" if a.tmc else "tvc"
    print(f"dims={a.dims} mode={a.mode} {a.dtype} {what}: {ms:.3f} ms  {nbytes / ms / 1e6:.1f} GB/s")


if __name__ == "__main__":
    main()
