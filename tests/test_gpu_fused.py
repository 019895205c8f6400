"""GPU parity of the fused forward (per-channel scale from folded batch
normalisation, shift, residual add, ReLU) and of the batch-norm folding
kernel, against the FP64 oracle on the same BF16/E4M3-rounded operands."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, make_inputs

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, TOL_F32, TOL_FP8, f64, oconv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _id(s):
    return f"{s.layout}-{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}x{s.S}-s{s.stride}-p{s.pad}-d{s.dil}"


def _bn_params(K, seed):
    g = torch.Generator().manual_seed(seed)
    gamma = torch.rand(K, generator=g) + 0.5
    bn_beta = torch.randn(K, generator=g)
    mean = torch.randn(K, generator=g) * 0.1
    var = torch.rand(K, generator=g) + 0.5
    return gamma, bn_beta, mean, var


def _fused_case(sh, in_dtype, out_dtype, algo, seed, relu=True, in_place=False):
    """Folds a batch norm with the device kernel, runs the fused forward and
    returns the normalised error against the oracle's fused forward."""
    x, w, b, _ = make_inputs(sh, seed)
    K = sh.K
    gamma, bn_beta, mean, var = _bn_params(K, seed + 1)
    dev = "cuda"
    scale, shift = F.bn_fold(gamma.to(dev), bn_beta.to(dev), mean.to(dev), var.to(dev), 1e-5,
                             bias=b.to(dev))
    p = oconv(sh)
    z = torch.randn(p.y_shape, generator=torch.Generator().manual_seed(seed + 2))
    xd, wd = x.to(in_dtype), w.to(in_dtype)
    zd = z.to(out_dtype)
    lay = sh.layout
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16 if in_dtype == torch.bfloat16 else B.GBCONV_F32,
                     B.GBCONV_BF16 if out_dtype == torch.bfloat16 else B.GBCONV_F32,
                     B.GBCONV_NHWC if lay == "NHWC" else B.GBCONV_NCHW)
    if algo is not None:
        bn = 256 if K > 128 else (64 if K <= 64 else 128)
        B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob, B.gbconv_config_t(bn, 0, 0, 0, algo)),
                "set_config")
    try:
        zg = zd.to(dev)
        out = zg if in_place else None
        y = F.conv2d_fused(xd.to(dev), wd.to(dev), shift, scale, zg, sh.stride, sh.pad, sh.dil,
                           relu, lay, out_dtype=out_dtype, out=out)
        F.device_error()
    finally:
        B.gbconv_shutdown()
    ref, bound = oracle.conv2d_fwd_fused(p, f64(xd), f64(wd), f64(scale), f64(shift), f64(zd),
                                         relu=relu, with_bound=True)
    return oracle.max_normalised_error(f64(y).reshape(-1), ref.reshape(-1), bound.reshape(-1))


TC_CASES = [
    (ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1), B.GBCONV_ALGO_IM2COL),
    (ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1), B.GBCONV_ALGO_SHIFT),
    (ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1), B.GBCONV_ALGO_SHIFT_T),
    (ConvShape(2, 64, 12, 12, 256, 1, 1, 1, 0, 1), B.GBCONV_ALGO_IM2COL),  # bottleneck end
    (ConvShape(2, 64, 12, 12, 256, 1, 1, 1, 0, 1), B.GBCONV_ALGO_SHIFT_T),
    (ConvShape(2, 128, 17, 15, 128, 3, 3, 2, 1, 1), B.GBCONV_ALGO_SHIFT_T),  # strided phases
    (ConvShape(2, 40, 10, 10, 72, 3, 3, 1, 1, 1), B.GBCONV_ALGO_IM2COL),   # K not a multiple of 32
    (ConvShape(2, 40, 10, 10, 72, 3, 3, 1, 1, 1), B.GBCONV_ALGO_SHIFT_T),
    (ConvShape(2, 32, 20, 30, 96, 3, 3, 1, 2, 2), None),                   # automatic choice
]


@pytest.mark.parametrize("sh,algo", TC_CASES, ids=[f"{_id(s)}-a{a}" for s, a in TC_CASES])
@pytest.mark.parametrize("out", ["bf16", "f32"])
def test_fused_bn_residual_relu_tensor_cores(sh, algo, out):
    od = torch.bfloat16 if out == "bf16" else torch.float32
    err = _fused_case(sh, torch.bfloat16, od, algo, seed=80)
    assert err <= (TOL_BF16_OUT if out == "bf16" else TOL_ACC32), err


@pytest.mark.parametrize("algo", [B.GBCONV_ALGO_IM2COL, B.GBCONV_ALGO_SHIFT_T])
def test_fused_residual_in_place(algo):
    """residual == y: every element is read before it is overwritten."""
    sh = ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1)
    err = _fused_case(sh, torch.bfloat16, torch.bfloat16, algo, seed=81, in_place=True)
    assert err <= TOL_BF16_OUT, err


@pytest.mark.parametrize("sh", [ConvShape(2, 5, 9, 8, 7, 3, 3, 1, 1, 1, "NCHW"),
                                ConvShape(2, 6, 9, 7, 5, 3, 3, 2, 1, 1, "NHWC")], ids=_id)
def test_fused_fp32_cuda_cores(sh):
    err = _fused_case(sh, torch.float32, torch.float32, None, seed=82)
    assert err <= TOL_F32, err


def test_fused_fp8():
    sh = ConvShape(2, 128, 10, 10, 128, 3, 3, 1, 1, 1)
    x, w, b, _ = make_inputs(sh, 83, "relu_normal", "he")
    dev = "cuda"
    xq, xs = F.quantize_e4m3(x.to(dev), rows=1)
    wq, ws = F.quantize_e4m3(w.to(dev), rows=sh.K)
    p = oconv(sh)
    g = torch.Generator().manual_seed(84)
    scale = (torch.rand(sh.K, generator=g) + 0.5).to(dev)
    z = torch.randn(p.y_shape, generator=g).bfloat16()
    y = F.conv2d_fused(xq, wq, b.to(dev), scale, z.to(dev), sh.stride, sh.pad, sh.dil, relu=True,
                       out_dtype=torch.bfloat16, x_scale=xs, w_scale=ws)
    F.device_error()
    xd = oracle.e4m3_to_f64(xq.view(torch.uint8).cpu().numpy()) * float(xs.item())
    wd = oracle.e4m3_to_f64(wq.view(torch.uint8).cpu().numpy()) * \
        ws.cpu().double().numpy()[:, None, None, None]
    ref, bound = oracle.conv2d_fwd_fused(p, xd, wd, f64(scale), f64(b), f64(z), relu=True,
                                         with_bound=True)
    err = oracle.max_normalised_error(f64(y).reshape(-1), ref.reshape(-1), bound.reshape(-1))
    assert err <= TOL_BF16_OUT, err
    ref2, bound2 = oracle.conv2d_fwd_fused(p, f64(x), f64(w), f64(scale), f64(b), f64(z),
                                           relu=True, with_bound=True)
    err2 = oracle.max_normalised_error(f64(y).reshape(-1), ref2.reshape(-1), bound2.reshape(-1))
    assert err2 <= TOL_FP8, err2


def test_fused_defaults_equal_plain_forward_bitwise():
    """No scale and no residual: the fused entry point is the plain forward."""
    sh = ConvShape(2, 64, 9, 11, 96, 3, 3, 1, 1, 1)
    x, w, b, _ = make_inputs(sh, 85)
    xd, wd, bd = x.bfloat16().cuda(), w.bfloat16().cuda(), b.cuda()
    y0 = F.conv2d(xd, wd, bd, 1, 1, 1, True)
    y1 = F.conv2d_fused(xd, wd, bd, None, None, 1, 1, 1, True)
    F.device_error()
    assert torch.equal(y0, y1)


def test_bn_fold_kernel_matches_oracle():
    K = 300
    gamma, bn_beta, mean, var = _bn_params(K, 86)
    bias = torch.randn(K, generator=torch.Generator().manual_seed(87))
    dev = "cuda"
    for b in (bias, None):
        s, t = F.bn_fold(gamma.to(dev), bn_beta.to(dev), mean.to(dev), var.to(dev), 1e-3,
                         bias=b.to(dev) if b is not None else None)
        F.device_error()
        a_ref, b_ref = oracle.bn_fold(gamma.double(), bn_beta.double(), mean.double(),
                                      var.double(), float(np.float32(1e-3)),
                                      bias=b.double() if b is not None else None)
        # FP32 with correctly rounded sqrt and division: a few ulps from FP64
        assert np.max(np.abs(f64(s) - a_ref) / np.abs(a_ref)) < 4e-7
        assert np.max(np.abs(f64(t) - b_ref) / (np.abs(bn_beta.double().numpy()) +
                                               np.abs(a_ref) * (np.abs(mean.double().numpy()) +
                                               (np.abs(b.double().numpy()) if b is not None else 0)))) < 1e-6


def test_fused_argument_checks():
    sh = ConvShape(1, 16, 8, 8, 16, 3, 3, 1, 1, 1)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1)
    x = torch.zeros(sh.x_shape(), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(sh.w_shape(), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(sh.y_shape(), dtype=torch.bfloat16, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # the residual may not be an input
    assert B.conv2d_fwd_fused(prob, x.data_ptr(), w.data_ptr(), 0, 0, x.data_ptr(), 0, 0,
                              y.data_ptr(), 0, 0, st) == B.GBCONV_ERR_INVALID_ARG
    # a misaligned residual is refused on the tensor-core path
    zz = torch.zeros(y.numel() + 8, dtype=torch.bfloat16, device="cuda")
    assert B.conv2d_fwd_fused(prob, x.data_ptr(), w.data_ptr(), 0, 0, zz.data_ptr() + 2, 0, 0,
                              y.data_ptr(), 0, 0, st) == B.GBCONV_ERR_ALIGNMENT
    assert B.gbconv_bn_fold(-1, 0, 0, 0, 0, 1e-5, 0, 0, 0, st) == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_bn_fold(0, 0, 0, 0, 0, 1e-5, 0, 0, 0, st) == B.GBCONV_OK
