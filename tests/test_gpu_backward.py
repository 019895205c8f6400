"""GPU parity of the backward passes (data gradient, weight and bias gradient)
and of the autograd Function, against the FP64 oracle's analytic gradients
(which the CPU suite pins to central finite differences)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import (ConvShape, config_backward, config_backward_fd,
                                          make_inputs)

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, TOL_F32, f64, oconv, sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _id(s):
    return f"{s.layout}-{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}x{s.S}-s{s.stride}-p{s.pad}-d{s.dil}"


def _grads(sh, dtype, seed, out_dtype=torch.float32, idx_dx=None, idx_dw=None):
    x, w, b, g = make_inputs(sh, seed, grad=True)
    dev = "cuda"
    xg, wg, gg = (x, w, g) if dtype == torch.float32 else (x.to(dtype), w.to(dtype), g.to(dtype))
    dx = F.conv2d_dgrad(gg.to(dev), wg.to(dev), tuple(x.shape), sh.stride, sh.pad, sh.dil,
                        sh.layout, out_dtype=out_dtype)
    dw, db = F.conv2d_wgrad(xg.to(dev), gg.to(dev), tuple(w.shape), sh.stride, sh.pad, sh.dil,
                            sh.layout)
    F.device_error()
    p = oconv(sh)
    dxr, dxb = oracle.conv2d_dgrad(p, f64(gg), f64(wg), idx=idx_dx, with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(xg), f64(gg), idx=idx_dw, with_bound=True)
    dbr, dbb = oracle.conv2d_bgrad(p, f64(gg), with_bound=True)
    gdx = f64(dx).reshape(-1)
    gdw = f64(dw).reshape(-1)
    if idx_dx is not None:
        gdx = gdx[idx_dx]
    if idx_dw is not None:
        gdw = gdw[idx_dw]
    return dict(dx=oracle.max_normalised_error(gdx, dxr.reshape(-1), dxb.reshape(-1)),
                dw=oracle.max_normalised_error(gdw, dwr.reshape(-1), dwb.reshape(-1)),
                db=oracle.max_normalised_error(f64(db), dbr, dbb))


BWD_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),          # tensor-core dgrad
    ConvShape(2, 32, 8, 8, 48, 1, 1, 1, 0, 1),
    ConvShape(1, 16, 12, 12, 24, 3, 3, 1, 2, 2),         # dilation 2, pad' = 2
    ConvShape(2, 24, 10, 10, 16, 5, 5, 1, 1, 1),         # pad < d(R-1): asymmetric rotation pad
    ConvShape(2, 32, 11, 11, 32, 3, 3, 2, 1, 1),         # stride 2: sub-pixel phase dgrad
    ConvShape(2, 8, 9, 7, 16, 3, 2, (2, 1), (1, 0), (1, 2)),
]


@pytest.mark.parametrize("sh", BWD_SHAPES, ids=_id)
def test_bf16_backward_small(sh):
    e = _grads(sh, torch.bfloat16, seed=30)
    assert e["dx"] <= TOL_ACC32 and e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


@pytest.mark.parametrize("sh", BWD_SHAPES[:2], ids=_id)
def test_bf16_dgrad_bf16_out(sh):
    e = _grads(sh, torch.bfloat16, seed=31, out_dtype=torch.bfloat16)
    assert e["dx"] <= TOL_BF16_OUT, e


# Data gradient of strided (or over-padded) BF16 NHWC layers: one stride-1
# band-kernel launch per sub-pixel phase of dx, zero fill for phases no tap reaches.
PHASE_DGRAD_SHAPES = [
    ConvShape(2, 128, 17, 15, 128, 3, 3, 2, 1, 1),    # ragged, 4 phases with 1-4 taps
    ConvShape(2, 64, 14, 13, 96, 1, 1, 2, 0, 1),      # 1x1 stride 2: 3 of 4 phases zero
    ConvShape(1, 64, 23, 19, 64, 5, 5, 2, 2, 1),      # offsets -1..1 in each phase
    ConvShape(1, 48, 21, 21, 64, 3, 3, 2, 2, 2),      # stride 2, dilation 2: odd phases zero
    ConvShape(1, 64, 25, 25, 32, 3, 3, 3, 1, 1),      # stride 3: 9 phases of one tap
    ConvShape(1, 32, 12, 12, 200, 3, 3, 2, 1, 1),     # 32 output channels, 200 reduction channels
    ConvShape(1, 192, 10, 10, 64, 3, 3, 2, 1, 1),     # 192 output channels: two channel tiles
    ConvShape(1, 32, 9, 9, 32, 3, 3, 1, 3, 1),        # stride 1, pad > d(R-1)
    ConvShape(2, 32, 9, 16, 48, 3, 3, (2, 1), 1, 1),  # row stride only
]


@pytest.mark.parametrize("sh", PHASE_DGRAD_SHAPES, ids=_id)
@pytest.mark.parametrize("out", ["f32", "bf16"])
def test_bf16_dgrad_subpixel_phases(sh, out):
    x, w, _, g = make_inputs(sh, 33, grad=True)
    od = torch.float32 if out == "f32" else torch.bfloat16
    wg, gg = w.bfloat16(), g.bfloat16()
    dx = F.conv2d_dgrad(gg.cuda(), wg.cuda(), tuple(x.shape), sh.stride, sh.pad, sh.dil, "NHWC",
                        out_dtype=od)
    F.device_error()
    ref, bound = oracle.conv2d_dgrad(oconv(sh), f64(gg), f64(wg), with_bound=True)
    err = oracle.max_normalised_error(f64(dx).reshape(-1), ref.reshape(-1), bound.reshape(-1))
    assert err <= (TOL_ACC32 if out == "f32" else TOL_BF16_OUT), err


def test_dgrad_subpixel_integer_exact():
    """Integer operands: every partial sum is exact in FP32, so the phase
    kernel must reproduce the oracle bit for bit (stride 2, 3x3, FP32 out)."""
    sh = ConvShape(2, 64, 15, 13, 64, 3, 3, 2, 1, 1)
    gen = torch.Generator().manual_seed(34)
    P, Q = sh.P, sh.Q
    g = torch.randint(-4, 5, (sh.N, P, Q, sh.K), generator=gen).float()
    w = torch.randint(-4, 5, (sh.K, sh.R, sh.S, sh.C), generator=gen).float()
    dx = F.conv2d_dgrad(g.bfloat16().cuda(), w.bfloat16().cuda(), (sh.N, sh.H, sh.W, sh.C),
                        sh.stride, sh.pad, sh.dil, "NHWC", out_dtype=torch.float32)
    F.device_error()
    ref = oracle.conv2d_dgrad(oconv(sh), f64(g), f64(w))
    assert np.array_equal(f64(dx).reshape(-1), np.asarray(ref).reshape(-1))


@pytest.mark.parametrize("sh", [ConvShape(2, 5, 9, 8, 7, 3, 3, 1, 1, 1, "NCHW"),
                                ConvShape(2, 5, 9, 8, 7, 3, 3, 2, 1, 1, "NHWC"),
                                ConvShape(1, 4, 11, 11, 3, 3, 3, 1, 2, 2, "NCHW"),
                                ConvShape(2, 3, 10, 9, 6, 2, 3, (2, 1), (0, 1), 1, "NCHW")],
                         ids=_id)
def test_fp32_backward_small(sh):
    e = _grads(sh, torch.float32, seed=32)
    assert e["dx"] <= TOL_F32 and e["dw"] <= TOL_F32 and e["db"] <= TOL_F32, e


def test_backward_fd_size():
    """The size on which the oracle's gradients are pinned to central finite
    differences: N=1, C=K=4, 6x6, 3x3 pad 1 (FP32 kernels)."""
    sh = config_backward_fd()
    for layout in ("NCHW", "NHWC"):
        sh.layout = layout
        e = _grads(sh, torch.float32, seed=33)
        assert max(e.values()) <= TOL_F32, e


def test_backward_full_size_sampled():
    """Backward workload: BF16 N=32, C=K=128, 56x56, 3x3 pad 1, g = N(0,1)."""
    sh = config_backward()
    nx = sh.N * sh.H * sh.W * sh.C
    nw = sh.K * sh.R * sh.S * sh.C
    e = _grads(sh, torch.bfloat16, seed=34, idx_dx=sampled(nx, 1000, 400),
               idx_dw=sampled(nw, 300, 401))
    assert e["dx"] <= TOL_ACC32 and e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


def test_wgrad_deterministic():
    sh = ConvShape(4, 64, 14, 14, 64, 3, 3, 1, 1, 1)
    x, w, b, g = make_inputs(sh, 35, grad=True)
    xb, gb = x.bfloat16().cuda(), g.bfloat16().cuda()
    dw1, db1 = F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
    dw2, db2 = F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
    F.device_error()
    assert torch.equal(dw1, dw2) and torch.equal(db1, db2)


@pytest.mark.parametrize("split", [1, 3, 64])
def test_wgrad_split_k_values(split):
    sh = ConvShape(2, 32, 12, 12, 48, 3, 3, 1, 1, 1)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_BF16,
                     B.GBCONV_BF16)
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob, B.gbconv_config_t(0, 0, split, 0)),
            "set_config")
    try:
        e = _grads(sh, torch.bfloat16, seed=36)
    finally:
        B.gbconv_shutdown()
    assert e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


def test_autograd_function():
    sh = ConvShape(2, 32, 10, 10, 64, 3, 3, 1, 1, 1)
    x, w, b, g = make_inputs(sh, 37, grad=True)
    dev = "cuda"
    xb = x.bfloat16().to(dev).requires_grad_()
    wb = w.bfloat16().to(dev).requires_grad_()
    bb = b.to(dev).requires_grad_()
    y = F.conv2d_autograd(xb, wb, bb, 1, 1, 1, False, "NHWC")
    y.backward(g.bfloat16().to(dev))
    F.device_error()
    p = oconv(sh)
    gd = f64(g.bfloat16())
    dxr, dxb = oracle.conv2d_dgrad(p, gd, f64(wb), with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(xb), gd, with_bound=True)
    dbr, dbb = oracle.conv2d_bgrad(p, gd, with_bound=True)
    # gradients come back in the parameters' dtype (bf16 rounding: 2^-9)
    assert oracle.max_normalised_error(f64(xb.grad), dxr, dxb) <= TOL_BF16_OUT
    assert oracle.max_normalised_error(f64(wb.grad), dwr, dwb) <= TOL_BF16_OUT
    assert oracle.max_normalised_error(f64(bb.grad), dbr, dbb) <= TOL_ACC32


def test_autograd_fp32_nchw():
    sh = ConvShape(1, 4, 6, 6, 4, 3, 3, 1, 1, 1, "NCHW")
    x, w, b, g = make_inputs(sh, 38, x_dist="uniform", w_dist="uniform", grad=True)
    dev = "cuda"
    xg, wg, bg = (t.to(dev).requires_grad_() for t in (x, w, b))
    y = F.conv2d_autograd(xg, wg, bg, 1, 1, 1, False, "NCHW")
    y.backward(g.to(dev))
    F.device_error()
    p = oconv(sh)
    dxr, dxb = oracle.conv2d_dgrad(p, f64(g), f64(w), with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(x), f64(g), with_bound=True)
    assert oracle.max_normalised_error(f64(xg.grad), dxr, dxb) <= TOL_F32
    assert oracle.max_normalised_error(f64(wg.grad), dwr, dwb) <= TOL_F32


# ---- tensor-core weight gradient (BF16 NHWC, C % 64 == 0) ----

TC_WGRAD_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),
    ConvShape(3, 128, 12, 12, 72, 3, 3, 2, 1, 1),     # partial output-channel tile, stride 2
    ConvShape(1, 64, 15, 13, 200, 3, 3, 1, 2, 2),     # two output-channel tiles, dilation 2
    ConvShape(2, 256, 7, 7, 64, 1, 1, 1, 0, 1),       # 256-channel tile, 1x1
    ConvShape(2, 192, 10, 10, 32, 5, 5, 1, 2, 1),     # 64-channel tiles, 5x5
    ConvShape(1, 64, 5, 5, 16, 3, 3, 1, 1, 1),        # fewer pixels than one 64-pixel step
]


@pytest.mark.parametrize("sh", TC_WGRAD_SHAPES, ids=_id)
def test_tc_wgrad_shapes(sh):
    e = _grads(sh, torch.bfloat16, seed=60)
    assert e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


@pytest.mark.parametrize("split", [1, 5, 16])
def test_tc_wgrad_split_values(split):
    sh = ConvShape(4, 128, 14, 14, 128, 3, 3, 1, 1, 1)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_BF16,
                     B.GBCONV_BF16)
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob, B.gbconv_config_t(0, 0, split, 0)),
            "set_config")
    try:
        e = _grads(sh, torch.bfloat16, seed=61)
    finally:
        B.gbconv_shutdown()
    assert e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


def test_tc_wgrad_integer_exact():
    """Integer x and g: all partial sums are integers below 2^24, so the
    tensor-core partials and the compensated slice sum are exact."""
    sh = ConvShape(2, 64, 10, 10, 96, 3, 3, 1, 1, 1)
    x, w, b, g = make_inputs(sh, 62, x_dist=("int", -4, 4), w_dist=("int", -4, 4), grad=True)
    g = torch.randint(-4, 5, g.shape, generator=torch.Generator().manual_seed(63)).float()
    xb, gb = x.bfloat16().cuda(), g.bfloat16().cuda()
    dw, db = F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
    F.device_error()
    p = oconv(sh)
    assert np.array_equal(f64(dw), oracle.conv2d_wgrad(p, f64(x), f64(g)))
    assert np.array_equal(f64(db), oracle.conv2d_bgrad(p, f64(g)))
