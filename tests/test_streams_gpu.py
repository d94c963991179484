"""tvc() on several streams and under CUDA-graph capture, checked against the
FP64 oracle.

tvc() takes its scratch (the split pieces of x for FP64, the partial sums of
a split n_k) per call from a stream-ordered pool, so two streams running it
at once must not disturb each other, and a captured call must replay with
the current contents of its inputs.  tvc_read_status synchronises, so it
must refuse to run on a stream under capture without breaking the capture.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

tg = pytest.importorskip("paper_2501_03121_gb300")

# (dims, mode, code): FP64 always uses scratch (split x); these shapes also
# split n_k over several blocks and keep partial sums there.
STREAM_CASES = [
    [((3, 300000), 1, oracle.F64), ((2, 5000, 9), 1, oracle.F64), ((3, 4099, 64), 1, oracle.F32)],
    [((20000, 64), 0, oracle.F64), ((6, 70, 33), 2, oracle.F64), ((2, 3, 250000), 2, oracle.F32)],
]


def _case(dims, mode, code, seed):
    A, Ao, _ = gu.inputs(dims, code, seed=seed)
    x = gu.vec(code, dims[mode], synth.stream_x(mode), seed=seed + 1)
    ref = oracle.tvc(Ao, mode, x)
    At, xt = gu.to_dev(A), gu.to_dev(x)
    y = torch.full(ref.shape, float("nan"), dtype=xt.dtype, device=gu.DEV)
    return At, xt, y, ref, Ao


def test_tvc_two_streams_concurrently():
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    work = []
    for si, cases in enumerate(STREAM_CASES):
        for ci, (dims, mode, code) in enumerate(cases):
            work.append((si, dims, mode, code) + _case(dims, mode, code, seed=10 * si + ci)[:4])
    torch.cuda.synchronize()
    # interleave the two streams' calls, several rounds, without ordering
    for _ in range(4):
        for si, dims, mode, code, At, xt, y, ref in work:
            with torch.cuda.stream(streams[si]):
                tg.tvc(At, mode, xt, y=y, shape=dims, stream=streams[si])
    torch.cuda.synchronize()
    for si, dims, mode, code, At, xt, y, ref in work:
        err = gu.rel_l2(y.cpu().numpy(), ref)
        assert err <= gu.TOL[code], (si, dims, mode, err)


@pytest.mark.parametrize("dims,mode,code", [((3, 300000), 1, oracle.F64), ((2, 3, 250000), 2, oracle.F32),
                                            ((40, 37, 66), 1, oracle.F64)])
def test_tvc_graph_capture_after_warm_call(dims, mode, code):
    At, xt, y, ref, A_host = _case(dims, mode, code, seed=3)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        tg.tvc(At, mode, xt, y=y, shape=dims, stream=s)  # warm call outside the capture
        with torch.cuda.graph(g, stream=s):
            tg.tvc(At, mode, xt, y=y, shape=dims, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert gu.rel_l2(y.cpu().numpy(), ref) <= gu.TOL[code]
    # new contents of x, same buffers: the replay must use them
    x2 = gu.vec(code, dims[mode], synth.stream_x(mode), seed=77)
    xt.copy_(torch.from_numpy(x2))
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert gu.rel_l2(y.cpu().numpy(), oracle.tvc(A_host, mode, x2)) <= gu.TOL[code]


def test_read_status_refuses_capture_and_keeps_it_valid():
    dims, mode, code = (3, 300000), 1, oracle.F64
    At, xt, y, ref, _ = _case(dims, mode, code, seed=5)
    status = torch.zeros(1, dtype=torch.int32, device=gu.DEV)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.stream(s):
        tg.tvc(At, mode, xt, y=y, shape=dims, stream=s)
        with torch.cuda.graph(g, stream=s):
            try:
                tg.read_status(status, stream=s)
            except tg.TVCError as e:
                refused = e.status
            tg.tvc(At, mode, xt, y=y, shape=dims, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    assert refused == 1  # TVC_ERR_INVALID_ARG, before touching the stream
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert gu.rel_l2(y.cpu().numpy(), ref) <= gu.TOL[code]
    assert tg.read_status(status) == 0
