"""GPU parity of the grouped (many problems, one persistent launch) forward,
including replay from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, grouped_problems, make_inputs

from _gpu_helpers import TOL_BF16, TOL_BF16_OUT, f64, oconv, sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _inputs(shapes, seed0):
    xs, ws, bs, masters = [], [], [], []
    for i, sh in enumerate(shapes):
        x, w, b, _ = make_inputs(sh, seed0 + i)
        xs.append(x.bfloat16().cuda())
        ws.append(w.bfloat16().cuda())
        bs.append(b.cuda())
        masters.append((x, w, b))
    return xs, ws, bs, masters


def _check(shapes, xs, ws, bs, masters, ys, relu, max_points=None, full_below_flops=0):
    """Every output of problems under `full_below_flops`, else `max_points`
    seeded samples (every output when max_points is None)."""
    for i, sh in enumerate(shapes):
        p = oconv(sh)
        idx = None
        total = int(np.prod(sh.y_shape()))
        if max_points is not None and total > max_points and sh.flops >= full_below_flops:
            idx = sampled(total, max_points, seed=500 + i)
        got = f64(ys[i]).reshape(-1)
        if idx is not None:
            got = got[idx]
        ref, bound = oracle.conv2d_fwd(p, f64(xs[i]), f64(ws[i]), f64(bs[i]), relu, idx=idx,
                                       with_bound=True)
        e = oracle.max_normalised_error(got, ref.reshape(-1), bound.reshape(-1))
        assert e <= TOL_BF16_OUT, (i, sh, e)
        x, w, b = masters[i]
        ref2, bound2 = oracle.conv2d_fwd(p, f64(x), f64(w), f64(b), relu, idx=idx,
                                         with_bound=True)
        e2 = oracle.max_normalised_error(got, ref2.reshape(-1), bound2.reshape(-1))
        assert e2 <= TOL_BF16, (i, sh, e2)


SMALL = [
    ConvShape(2, 64, 9, 9, 64, 3, 3, 1, 1, 1),
    ConvShape(1, 16, 14, 14, 32, 1, 1, 1, 0, 1),
    ConvShape(3, 128, 7, 7, 256, 3, 3, 1, 1, 1),
    ConvShape(2, 32, 15, 15, 48, 5, 5, 2, 2, 1),
    ConvShape(1, 48, 28, 28, 16, 7, 7, 2, 3, 1),
    ConvShape(4, 256, 4, 4, 128, 1, 1, 1, 0, 1),
]


def test_grouped_small():
    xs, ws, bs, masters = _inputs(SMALL, 600)
    strides = [s.stride for s in SMALL]
    pads = [s.pad for s in SMALL]
    ys = F.conv2d_grouped(xs, ws, bs, strides, pads, relu=True)
    F.device_error()
    _check(SMALL, xs, ws, bs, masters, ys, relu=True)


def test_grouped_matches_single_launches_bitwise():
    """The grouped launch runs the im2col kernel body; single launches forced
    onto the same algorithm and tile width reproduce it bit for bit."""
    xs, ws, bs, _ = _inputs(SMALL, 610)
    ys = F.conv2d_grouped(xs, ws, bs, [s.stride for s in SMALL], [s.pad for s in SMALL])
    try:
        for i, sh in enumerate(SMALL):
            prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, 1,
                             B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS)
            s, cfg = B.gbconv_get_config(B.GBCONV_OP_FWD, prob)
            cfg.algo = B.GBCONV_ALGO_IM2COL
            B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob, cfg), "set_config")
            y1 = F.conv2d(xs[i], ws[i], bs[i], sh.stride, sh.pad, 1, False, "NHWC")
            F.device_error()
            assert torch.equal(y1, ys[i]), i
    finally:
        B.gbconv_shutdown()


def test_grouped_workload_64_problems_graph():
    """The 64-problem workload (shapes drawn from seed 1, committed JSON), one
    persistent launch captured in a CUDA graph and replayed; every output of
    each problem under 1 GFLOP and 4096 seeded outputs of the larger ones
    against the oracle."""
    shapes = grouped_problems()
    assert len(shapes) == 64
    xs, ws, bs, masters = _inputs(shapes, 1000)
    ys = [torch.empty(s.y_shape(), dtype=torch.bfloat16, device="cuda") for s in shapes]
    strides = [s.stride for s in shapes]
    pads = [s.pad for s in shapes]
    F.conv2d_grouped(xs, ws, bs, strides, pads, relu=True, outs=ys)  # warm-up (sets attributes)
    torch.cuda.synchronize()
    for y in ys:
        y.fill_(0)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            F.conv2d_grouped(xs, ws, bs, strides, pads, relu=True, outs=ys)
    graph.replay()
    torch.cuda.synchronize()
    F.device_error()
    _check(shapes, xs, ws, bs, masters, ys, relu=True, max_points=4096, full_below_flops=1e9)


def test_grouped_tuned_tile_widths_match_oracle():
    """Each problem tuned as the grouped launch's body (gbconv_tune with
    GBCONV_OP_GROUPED) stores one of the candidate tile widths; the grouped
    launch then runs with the stored widths and still matches the oracle."""
    xs, ws, bs, masters = _inputs(SMALL, 620)
    ys = [torch.empty(s.y_shape(), dtype=torch.bfloat16, device="cuda") for s in SMALL]
    st = torch.cuda.current_stream().cuda_stream
    try:
        for i, sh in enumerate(SMALL):
            prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, 1,
                             B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC,
                             B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU)
            s, c = B.gbconv_tune(B.GBCONV_OP_GROUPED, prob, xs[i].data_ptr(), ws[i].data_ptr(),
                                 bs[i].data_ptr(), ys[i].data_ptr(), 0, 0, 2, st)
            B.check(s, "gbconv_tune")
            assert c.block_n in (32, 64, 128, 256)
            s, c2 = B.gbconv_get_config(B.GBCONV_OP_GROUPED, prob)
            assert s == B.GBCONV_OK and c2.block_n == c.block_n
        out = F.conv2d_grouped(xs, ws, bs, [s.stride for s in SMALL], [s.pad for s in SMALL],
                               relu=True)
        F.device_error()
    finally:
        B.gbconv_shutdown()
    _check(SMALL, xs, ws, bs, masters, out, relu=True)
