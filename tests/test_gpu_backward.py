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

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, TOL_F32, f64, oconv

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


def test_backward_full_size_every_output():
    """Backward workload: BF16 N=32, C=K=128, 56x56, 3x3 pad 1, g = N(0,1).
    Every element of dx (12.8 M), dw (147 456) and db against the oracle."""
    sh = config_backward()
    e = _grads(sh, torch.bfloat16, seed=34)
    assert e["dx"] <= TOL_ACC32 and e["dw"] <= TOL_ACC32 and e["db"] <= TOL_ACC32, e


def test_backward_full_size_bf16_dx_every_output():
    """The same workload with dx in BF16 (the dtype autograd hands back)."""
    sh = config_backward()
    e = _grads(sh, torch.bfloat16, seed=35, out_dtype=torch.bfloat16)
    assert e["dx"] <= TOL_BF16_OUT, e


def test_strided_dgrad_full_size_every_output():
    """Data gradient of the 3x3 stride-2 ResNet layer (128 -> 128, 56 -> 28,
    batch 32) by sub-pixel phases: every element of dx."""
    from paper_2207_00257_gb300.synth import resnet_layers
    sh = resnet_layers(32)[3]
    x, w, _, g = make_inputs(sh, 36, grad=True)
    wg, gg = w.bfloat16(), g.bfloat16()
    dx = F.conv2d_dgrad(gg.cuda(), wg.cuda(), tuple(x.shape), sh.stride, sh.pad, sh.dil, "NHWC",
                        out_dtype=torch.float32)
    F.device_error()
    ref, bound = oracle.conv2d_dgrad(oconv(sh), f64(gg), f64(wg), with_bound=True)
    err = oracle.max_normalised_error(f64(dx).reshape(-1), ref.reshape(-1), bound.reshape(-1))
    assert err <= TOL_ACC32, err


# ---- the gradient through ReLU (gbconv_relu_grad) ----

_DTS = (torch.float32, torch.bfloat16)


@pytest.mark.parametrize("yd", _DTS, ids=["yf32", "ybf16"])
@pytest.mark.parametrize("gd", _DTS, ids=["gf32", "gbf16"])
@pytest.mark.parametrize("od", _DTS, ids=["of32", "obf16"])
@pytest.mark.parametrize("n", [1, 7, 8, 4099, 300000])
def test_relu_grad_kernel_bitwise(yd, gd, od, n):
    """g_out = g where y > 0 else 0, bit for bit the oracle's definition
    (then rounded to BF16 by the oracle's quantiser for BF16 outputs). y holds
    exact zeros (ReLU outputs), negative values and -0.0."""
    gen = torch.Generator().manual_seed(90 + n)
    y = torch.randn(n, generator=gen).clamp_min(0.0)
    y[1::7] = -torch.rand(len(range(1, n, 7)), generator=gen)
    if n > 3:
        y[3] = -0.0
    g = torch.randn(n, generator=gen) * 3
    yy, gg = y.to(yd), g.to(gd)
    out = F.relu_grad(yy.cuda(), gg.cuda(), out_dtype=od)
    F.device_error()
    ref = oracle.relu_grad(f64(yy), f64(gg))
    if od == torch.bfloat16:
        ref = oracle.round_bf16(ref)
    else:
        ref = ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(f64(out), ref)


def test_relu_grad_in_place_and_unaligned():
    """In place (g_out = g), and views one element off the 16-byte boundary
    (the scalar path)."""
    gen = torch.Generator().manual_seed(95)
    n = 10001
    y = torch.randn(n + 1, generator=gen).bfloat16().cuda()
    g = torch.randn(n + 1, generator=gen).bfloat16().cuda()
    ref = oracle.relu_grad(f64(y), f64(g))
    g2 = g.clone()
    F.relu_grad(y, g2, out=g2)
    F.device_error()
    assert np.array_equal(f64(g2), ref)
    out = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    F.relu_grad(y[1:], g[1:], out_dtype=torch.float32, out=out[1:])
    F.device_error()
    assert np.array_equal(f64(out[1:]), ref[1:])


def test_relu_grad_rejects_overlap():
    y = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    g = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    s = B.gbconv_relu_grad(y.data_ptr(), B.GBCONV_BF16, g.data_ptr(), B.GBCONV_BF16,
                           y.data_ptr(), B.GBCONV_BF16, 64, st)
    assert s == B.GBCONV_ERR_INVALID_ARG
    s = B.gbconv_relu_grad(y.data_ptr(), B.GBCONV_BF16, g.data_ptr(), B.GBCONV_BF16,
                           g.data_ptr() + 2, B.GBCONV_BF16, 32, st)
    assert s == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_relu_grad(y.data_ptr(), B.GBCONV_E4M3, g.data_ptr(), B.GBCONV_BF16,
                              g.data_ptr(), B.GBCONV_BF16, 64, st) == B.GBCONV_ERR_UNSUPPORTED


def _relu_case(sh, dtype, seed):
    """Integer x, w and half-integer b: every pre-activation z is k + 1/2, so
    the ReLU mask (z > 0) is the same on both sides whatever the rounding."""
    gen = torch.Generator().manual_seed(seed)
    x = torch.randint(-3, 4, sh.x_shape(), generator=gen).float()
    w = torch.randint(-3, 4, sh.w_shape(), generator=gen).float()
    b = torch.randint(-4, 4, (sh.K,), generator=gen).float() + 0.5
    g = torch.randn(sh.y_shape(), generator=gen)
    dev = "cuda"
    xg = x.to(dtype).to(dev).requires_grad_()
    wg = w.to(dtype).to(dev).requires_grad_()
    bg = b.to(dev).requires_grad_()
    y = F.conv2d_autograd(xg, wg, bg, sh.stride, sh.pad, sh.dil, True, sh.layout)
    gd = g.to(y.dtype)
    y.backward(gd.to(dev))
    F.device_error()
    p = oconv(sh)
    z = oracle.conv2d_fwd(p, f64(x), f64(w), f64(b))
    assert np.min(np.abs(z)) >= 0.5 and np.any(z < 0) and np.any(z > 0)
    gz = oracle.relu_grad(np.maximum(z, 0.0), f64(gd))
    dxr, dxb = oracle.conv2d_dgrad(p, gz, f64(w), with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(x), gz, with_bound=True)
    dbr, dbb = oracle.conv2d_bgrad(p, gz, with_bound=True)
    return (oracle.max_normalised_error(f64(xg.grad), dxr, dxb),
            oracle.max_normalised_error(f64(wg.grad), dwr, dwb),
            oracle.max_normalised_error(f64(bg.grad), dbr, dbb))


def test_autograd_relu_bf16_matches_oracle():
    """relu=True through Conv2dFn: the library masks the upstream gradient
    (gbconv_relu_grad) and runs dgrad / wgrad; against the oracle's analytic
    gradient of sum g * relu(conv(x, w) + b)."""
    ex, ew, eb = _relu_case(ConvShape(2, 32, 10, 10, 64, 3, 3, 1, 1, 1), torch.bfloat16, 39)
    # dx and dw come back in BF16 (rounding 2^-9), db in fp32
    assert ex <= TOL_BF16_OUT and ew <= TOL_BF16_OUT and eb <= TOL_ACC32, (ex, ew, eb)


def test_autograd_relu_fp32_nchw_strided_matches_oracle():
    ex, ew, eb = _relu_case(ConvShape(2, 6, 9, 8, 5, 3, 3, 2, 1, 1, "NCHW"), torch.float32, 40)
    assert ex <= TOL_F32 and ew <= TOL_F32 and eb <= TOL_F32, (ex, ew, eb)


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


# ---- the two tensor-core weight-gradient kernels, forced in turn ----

BAND_WGRAD_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),
    ConvShape(1, 64, 15, 13, 200, 3, 3, 1, 2, 2),      # dilation 2, two output-channel tiles
    ConvShape(2, 192, 10, 10, 32, 5, 5, 1, 2, 1),      # 5x5, three 64-channel input tiles
    ConvShape(1, 64, 5, 5, 16, 3, 3, 1, 1, 1),         # fewer positions than one band
    ConvShape(1, 64, 9, 10, 64, 3, 3, 1, 1, 2),        # pad < (S-1)*dil: row width Q + 3
    ConvShape(1, 64, 9, 10, 40, 3, 3, 1, (1, 0), 1),   # no column padding: no wrap
    ConvShape(1, 64, 9, 10, 64, 3, 3, 1, (0, 2), 1),   # column padding 2
    ConvShape(2, 128, 5, 70, 136, 3, 3, 1, 1, 1),      # ragged second output-channel tile
    ConvShape(1, 256, 6, 6, 64, 3, 3, 1, 1, 1),        # two 128-channel input tiles
    ConvShape(1, 64, 4, 4, 8, 2, 2, 1, 0, 1),          # 2x2, K = 8
    ConvShape(1, 64, 6, 20, 64, 1, 7, 1, 3, 1),        # 1x7
    ConvShape(1, 128, 7, 6, 64, 5, 3, 1, 3, 1),        # 5x3, pad 3
]


def _wgrad_err(sh, seed, algo, split=0):
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, B.GBCONV_BF16)
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob, B.gbconv_config_t(0, 0, split, 0, algo)),
            "set_config")
    try:
        x, _, _, g = make_inputs(sh, seed, grad=True)
        xb, gb = x.bfloat16(), g.bfloat16()
        dw, db = F.conv2d_wgrad(xb.cuda(), gb.cuda(), (sh.K, sh.R, sh.S, sh.C), sh.stride, sh.pad,
                                sh.dil)
        F.device_error()
    finally:
        B.gbconv_shutdown()
    p = oconv(sh)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(xb), f64(gb), with_bound=True)
    dbr, dbb = oracle.conv2d_bgrad(p, f64(gb), with_bound=True)
    return (oracle.max_normalised_error(f64(dw).reshape(-1), dwr.reshape(-1), dwb.reshape(-1)),
            oracle.max_normalised_error(f64(db), dbr, dbb))


@pytest.mark.parametrize("algo", ["band", "im2col"])
@pytest.mark.parametrize("sh", BAND_WGRAD_SHAPES, ids=_id)
def test_wgrad_band_and_per_tap_kernels(sh, algo):
    a = B.GBCONV_ALGO_SHIFT if algo == "band" else B.GBCONV_ALGO_IM2COL
    for split in (0, 3):
        ew, eb = _wgrad_err(sh, 64, a, split)
        assert ew <= TOL_ACC32 and eb <= TOL_ACC32, (split, ew, eb)


@pytest.mark.parametrize("algo", ["band", "im2col"])
def test_wgrad_kernels_integer_exact(algo):
    """Integer x and g on both tensor-core kernels, ragged bands and tiles."""
    sh = ConvShape(3, 128, 11, 13, 72, 3, 3, 1, 1, 1)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_BF16,
                     B.GBCONV_BF16)
    a = B.GBCONV_ALGO_SHIFT if algo == "band" else B.GBCONV_ALGO_IM2COL
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob, B.gbconv_config_t(0, 0, 7, 0, a)),
            "set_config")
    try:
        x, w, _, g = make_inputs(sh, 65, x_dist=("int", -4, 4), w_dist=("int", -4, 4), grad=True)
        g = torch.randint(-4, 5, g.shape, generator=torch.Generator().manual_seed(66)).float()
        dw, db = F.conv2d_wgrad(x.bfloat16().cuda(), g.bfloat16().cuda(), tuple(w.shape), 1, 1, 1)
        F.device_error()
    finally:
        B.gbconv_shutdown()
    p = oconv(sh)
    assert np.array_equal(f64(dw), oracle.conv2d_wgrad(p, f64(x), f64(g)))
    assert np.array_equal(f64(db), oracle.conv2d_bgrad(p, f64(g)))


def test_wgrad_band_full_size_sampled():
    """The band kernel on the backward workload (N=32, C=K=128, 56x56, 3x3) at
    its default slice count: 4096 sampled weights and every bias."""
    sh = config_backward()
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_BF16,
                     B.GBCONV_BF16)
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob,
                                B.gbconv_config_t(0, 0, 0, 0, B.GBCONV_ALGO_SHIFT)), "set_config")
    try:
        x, _, _, g = make_inputs(sh, 67, grad=True)
        xb, gb = x.bfloat16(), g.bfloat16()
        dw, db = F.conv2d_wgrad(xb.cuda(), gb.cuda(), (sh.K, sh.R, sh.S, sh.C), 1, 1, 1)
        F.device_error()
    finally:
        B.gbconv_shutdown()
    p = oconv(sh)
    idx = np.random.default_rng(68).choice(sh.K * sh.R * sh.S * sh.C, 4096, replace=False)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(xb), f64(gb), idx=idx, with_bound=True)
    assert oracle.max_normalised_error(f64(dw).reshape(-1)[idx], dwr, dwb) <= TOL_ACC32
    dbr, dbb = oracle.conv2d_bgrad(p, f64(gb), with_bound=True)
    assert oracle.max_normalised_error(f64(db), dbr, dbb) <= TOL_ACC32
