"""Full-size power-method workloads on the GPU against the FP64 oracle's
stored results (tests/golden/hopm_fullsize.json, written by
tests/golden/make_fullsize_hopm.py from the host generator and the oracle
only: oracle.quantise and oracle.hopm3, Algorithm 1).

The tensors are filled on the device by the generator that reproduces the
host generator's bits (checked element by element in test_tvc_gpu.py), so
the GPU runs on exactly the oracle's inputs.

* planted rank-1 + noise, 256^4 binary32 (2^32 elements: every index of the
  HOPM launch sequence past 2^32 is exercised), 50 sweeps, tol 1e-8, from a
  start that overlaps the planted factors: lambda of every sweep within 1e-5
  of the oracle (FP32 accumulation), final x_j within 2e-4, the subspace
  error against the planted factors equal to the oracle's.
* 2048^3 N(0,1) exp(U[-3,3]), 30 sweeps from all-ones: binary32 storage
  within 1e-5 of the oracle; BF16 and E4M3 per-slab storage (Section 5.5):
  the quantiser's codes and scales bit for bit equal to the oracle's (SHA-256
  over all 8.6e9 codes), lambda of every sweep within 1e-5 of the oracle on
  the same stored codes (kernel error), and the final lambda within 1e-3 of
  the oracle on the binary32 source (storage error).
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest
import torch

import synth
from tests import gpu_util as gu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

tg = pytest.importorskip("paper_2501_03121_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hopm_fullsize.json")


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def check_run(r, ref, hist_tol=1e-5, x_tol=2e-4, sweeps_slack=0):
    n = int(r.sweeps.item())
    assert abs(n - ref["sweeps"]) <= sweeps_slack, (n, ref["sweeps"])
    m = min(n, ref["sweeps"])
    hist = r.lam_hist.cpu().numpy()[:m]
    np.testing.assert_allclose(hist, ref["lam_hist"][:m], rtol=hist_tol)
    assert abs(r.lam.item() - ref["lam"]) <= hist_tol * ref["lam"]
    for xg, probe in zip(r.x, ref["x_probe"]):
        idx = torch.tensor([int(i) for i in probe], device=gu.DEV)
        got = xg[idx].cpu().numpy().astype(np.float64)
        want = np.array(list(probe.values()))
        assert np.max(np.abs(got - want)) <= x_tol, (got, want)


def sha256_dev(t):
    h = hashlib.sha256()
    flat = t.reshape(-1).view(torch.uint8)
    step = 1 << 30
    for lo in range(0, flat.numel(), step):
        h.update(flat[lo:lo + step].cpu().numpy())
    return h.hexdigest()


def test_planted_256_4_fp32_against_oracle():
    import synth.device as sd
    ref = golden()["planted"]
    dims = tuple(ref["dims"])
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    A = torch.empty(math.prod(dims), dtype=torch.float32, device=gu.DEV)
    sd.fill(A, "planted", 0, 0, dims=dims, us=us)
    xs = []
    for j, n in enumerate(dims):
        v = us[j] + synth.unit_gaussian(1, synth.stream_u(j), n)
        xs.append(torch.from_numpy((v / np.linalg.norm(v)).astype(np.float32)).to(gu.DEV))
    r = tg.hopm(A, xs, ref["iters"], ref["tol"], shape=dims)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    # The stopping sweep compares successive lambdas at 1e-8, below the FP32
    # rounding of the contractions, so it may differ by a sweep or two.
    check_run(r, ref, sweeps_slack=2)
    sub = max(math.sqrt(max(0.0, 1.0 - float(np.dot(x.cpu().numpy().astype(np.float64), u)) ** 2))
              for x, u in zip(r.x, us))
    assert abs(sub - ref["subspace_error"]) <= 1e-4, (sub, ref["subspace_error"])
    del A
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def mixed_source():
    import synth.device as sd
    ref = golden()["mixed"]
    dims = tuple(ref["dims"])
    src = torch.empty(math.prod(dims), dtype=torch.float32, device=gu.DEV)
    sd.fill(src, "lognormal", 0, synth.STREAM_A)
    yield ref, dims, src
    del src
    torch.cuda.empty_cache()


def _ones(dims):
    return [torch.full((n,), 1.0 / math.sqrt(n), dtype=torch.float32, device=gu.DEV) for n in dims]


def test_mixed_2048_3_fp32_against_oracle(mixed_source):
    ref, dims, src = mixed_source
    r = tg.hopm(src, _ones(dims), ref["iters"], shape=dims)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    check_run(r, ref["f32"])


@pytest.mark.parametrize("name", ["bf16", "e4m3"])
def test_mixed_2048_3_low_precision_lambda(mixed_source, name):
    ref, dims, src = mixed_source
    code = {"bf16": tg.BF16, "e4m3": tg.E4M3}[name]
    codes, scales, status = tg.quantise(src.view(dims), code)
    assert int(status.item()) == 0
    # the full-size quantiser equals the oracle's bit for bit
    assert sha256_dev(scales) == ref[name]["sha256_scales"]
    assert sha256_dev(codes) == ref[name]["sha256_codes"]
    r = tg.hopm(codes.view(-1), _ones(dims), ref["iters"], scales=scales, shape=dims)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    # kernel error: the oracle on the same stored codes
    check_run(r, ref[name])
    # storage error: the oracle on the binary32 source
    err = abs(r.lam.item() - ref["f32"]["lam"]) / ref["f32"]["lam"]
    print(f"{name} lambda relative error against the FP64 oracle on the source: {err:.3e}")
    assert err <= 1e-3
    del codes, scales, r
    torch.cuda.empty_cache()
