"""GPU parity of the forward with channel groups (tensor cores per group,
depthwise kernel, CUDA-core implicit GEMM per group) against the FP64
oracle's grouped convolution on the same rounded operands."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, TOL_F32, f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _case(N, C, H, W, K, R, S, st, pd, dl, G, layout, in_dtype, out_dtype, seed, fused=False,
          relu=True):
    p = oracle.Conv(N, C, H, W, K, R, S, st, pd, dl, layout, groups=G)
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(p.x_shape, generator=g).to(in_dtype)
    w = (torch.randn(p.w_shape, generator=g) / np.sqrt(C // G * R * S)).to(in_dtype)
    b = torch.rand(K, generator=g) * 0.2 - 0.1
    alpha = (torch.rand(K, generator=g) + 0.5) if fused else None
    z = torch.randn(p.y_shape, generator=g).to(out_dtype) if fused else None
    dev = "cuda"
    y = F.conv2d_fused(x.to(dev), w.to(dev), b.to(dev),
                       alpha.to(dev) if alpha is not None else None,
                       z.to(dev) if z is not None else None, st, pd, dl, relu, layout,
                       out_dtype=out_dtype, groups=G)
    F.device_error()
    ref, bound = oracle.conv2d_fwd_fused(p, f64(x), f64(w), f64(alpha) if fused else None, f64(b),
                                         f64(z) if fused else None, relu=relu, with_bound=True)
    return oracle.max_normalised_error(f64(y).reshape(-1), ref.reshape(-1), bound.reshape(-1))


# (N, C, H, W, K, R, S, stride, pad, dil, G)
TC_GROUPS = [
    (2, 128, 10, 11, 128, 3, 3, 1, 1, 1, 2),    # two 64-channel groups
    (2, 256, 9, 9, 128, 1, 1, 1, 0, 1, 4),      # 1x1, 64 -> 32 per group
    (1, 128, 12, 12, 128, 3, 3, 2, 1, 1, 8),    # 16 channels per group, stride 2
    (2, 96, 8, 9, 48, 5, 5, 1, 2, 1, 3),        # 32 -> 16 per group
]
DEPTHWISE = [
    (2, 64, 12, 11, 64, 3, 3, 1, 1, 1, 64),
    (2, 128, 15, 14, 128, 5, 5, 2, 2, 1, 128),
    (1, 32, 9, 9, 32, 3, 3, 1, 2, 2, 32),       # dilation 2
    (2, 16, 7, 6, 16, 7, 7, 1, 3, 1, 16),
]
SMALL_GROUPS = [  # C/G = K/G in {2, 4, 8}: the direct kernel of the depthwise case
    (2, 128, 8, 8, 128, 3, 3, 1, 1, 1, 32),     # 4 channels per group (ResNeXt-style)
    (1, 64, 9, 10, 64, 3, 3, 2, 1, 1, 32),      # 2 channels per group, stride 2
    (2, 64, 7, 9, 64, 5, 3, 1, (2, 1), 1, 8),   # 8 channels per group
    (2, 64, 9, 13, 64, 3, 3, 1, 1, 1, 32),      # 2 channels per group, unit stride
    (1, 32, 7, 10, 32, 3, 3, 1, (1, 2), 1, 16), # unit stride, horizontal padding 2
    (2, 128, 9, 11, 128, 3, 3, 2, 1, 1, 32),    # 4 channels per group, stride 2
]
DIRECT_BF16 = [  # rows too wide to stage two bands in shared memory: the direct kernel
    (1, 2048, 4, 24, 2048, 3, 3, 1, 1, 1, 2048),
    (1, 1024, 3, 40, 1024, 3, 3, 1, 1, 1, 256),  # 4 channels per group
    (1, 1024, 5, 30, 1024, 3, 3, 2, 1, 1, 512),  # 2 channels per group, stride 2
]
CUDA_CORE_GROUPS = [
    (2, 32, 9, 9, 64, 3, 3, 1, 1, 1, 32),       # depthwise with multiplier 2
    (1, 12, 7, 8, 18, 3, 2, (2, 1), (1, 0), 1, 6),
    (2, 48, 6, 6, 48, 3, 3, 1, 1, 1, 3),        # 16 channels per group
]


def _cid(c):
    return "x".join(str(v) for v in c)


@pytest.mark.parametrize("case", TC_GROUPS, ids=_cid)
@pytest.mark.parametrize("out", ["bf16", "f32"])
def test_groups_tensor_cores(case, out):
    od = torch.bfloat16 if out == "bf16" else torch.float32
    err = _case(*case, "NHWC", torch.bfloat16, od, seed=90)
    assert err <= (TOL_BF16_OUT if out == "bf16" else TOL_ACC32), err


@pytest.mark.parametrize("case", DEPTHWISE, ids=_cid)
@pytest.mark.parametrize("dt", ["bf16-bf16", "bf16-f32", "f32-f32"])
@pytest.mark.parametrize("fused", [False, True])
def test_depthwise(case, dt, fused):
    ind, outd = {"bf16-bf16": (torch.bfloat16, torch.bfloat16),
                 "bf16-f32": (torch.bfloat16, torch.float32),
                 "f32-f32": (torch.float32, torch.float32)}[dt]
    err = _case(*case, "NHWC", ind, outd, seed=91, fused=fused)
    tol = TOL_BF16_OUT if outd == torch.bfloat16 else (TOL_F32 if ind == torch.float32 else TOL_ACC32)
    assert err <= tol, err


@pytest.mark.parametrize("case", SMALL_GROUPS, ids=_cid)
@pytest.mark.parametrize("dt", ["bf16-bf16", "f32-f32"])
def test_small_groups_direct_kernel(case, dt):
    ind, outd = (torch.bfloat16, torch.bfloat16) if dt == "bf16-bf16" else (torch.float32, torch.float32)
    err = _case(*case, "NHWC", ind, outd, seed=94, fused=True)
    assert err <= (TOL_BF16_OUT if outd == torch.bfloat16 else TOL_F32), err


@pytest.mark.parametrize("case", DIRECT_BF16, ids=_cid)
@pytest.mark.parametrize("out", ["bf16", "f32"])
def test_groups_direct_kernel_wide_rows(case, out):
    od = torch.bfloat16 if out == "bf16" else torch.float32
    err = _case(*case, "NHWC", torch.bfloat16, od, seed=95, fused=True)
    assert err <= (TOL_BF16_OUT if out == "bf16" else TOL_ACC32), err


@pytest.mark.parametrize("case", CUDA_CORE_GROUPS + SMALL_GROUPS[:1], ids=_cid)
@pytest.mark.parametrize("layout", ["NHWC", "NCHW"])
def test_groups_cuda_cores(case, layout):
    ind = torch.bfloat16 if layout == "NHWC" else torch.float32
    err = _case(*case, layout, ind, torch.float32, seed=92, fused=True)
    assert err <= (TOL_ACC32 if ind == torch.bfloat16 else TOL_F32), err


# (N, C, HW, G): the bench's grouped layers at batch 32 (two blocks per SM,
# about six bands each), and a 256-channel depthwise layer whose two stages
# take one block per SM; both refill stages while the other band computes.
FULL_SIZE = [(32, 128, 56, 128), (32, 128, 56, 32), (8, 256, 56, 256)]


@pytest.mark.parametrize("N,C,HW,G", FULL_SIZE, ids=lambda v: str(v))
def test_groups_full_size_every_output(N, C, HW, G):
    p = oracle.Conv(N, C, HW, HW, C, 3, 3, 1, 1, 1, "NHWC", groups=G)
    g = torch.Generator().manual_seed(96)
    x = torch.randn(p.x_shape, generator=g).bfloat16()
    w = (torch.randn(p.w_shape, generator=g) / np.sqrt(C // G * 9)).bfloat16()
    b = torch.rand(C, generator=g) * 0.2 - 0.1
    y = F.conv2d(x.cuda(), w.cuda(), b.cuda(), 1, 1, 1, True, groups=G)
    F.device_error()
    ref, bound = oracle.conv2d_fwd(p, f64(x), f64(w), f64(b), True, with_bound=True)
    err = oracle.max_normalised_error(f64(y).reshape(-1), ref.reshape(-1), bound.reshape(-1))
    assert err <= TOL_BF16_OUT, err


def test_groups_with_fused_epilogue_on_tensor_core_shapes():
    """A tensor-core-shaped grouped layer with scale and residual runs the
    CUDA-core path (the grouped launch has no fused epilogue): same results."""
    err = _case(*TC_GROUPS[0], "NHWC", torch.bfloat16, torch.bfloat16, seed=93, fused=True)
    assert err <= TOL_BF16_OUT, err


def test_groups_argument_checks():
    st = torch.cuda.current_stream().cuda_stream
    bad = B.problem(1, 6, 5, 5, 4, 3, 3, groups=4)
    assert B.conv2d_fwd(bad, 16, 32, 0, 0, 0, 64, 0, 0, st) == B.GBCONV_ERR_INVALID_ARG
    p = B.problem(1, 64, 8, 8, 64, 3, 3, 1, 1, 1, groups=64)
    assert B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, p) == (B.GBCONV_OK, 0)
    s, nw = B.gbconv_workspace_size(B.GBCONV_OP_WGRAD, p)
    assert s == B.GBCONV_OK and nw > 0
    assert B.conv2d_wgrad(p, 16, 32, 64, 0, 0, 0, st) == B.GBCONV_ERR_WORKSPACE  # none given
    e4 = B.problem(1, 64, 8, 8, 64, 3, 3, 1, 1, 1, B.GBCONV_E4M3, B.GBCONV_BF16, groups=2)
    assert B.conv2d_fwd(e4, 16, 32, 0, 16, 16, 64, 0, 0, st) == B.GBCONV_ERR_UNSUPPORTED


# ---- gradients of grouped layers (CUDA cores, one grid layer per group) ----

GRAD_CASES = [  # (N, C, H, W, K, R, stride, pad, G)
    (2, 16, 9, 9, 16, 3, 1, 1, 16),     # depthwise
    (2, 16, 9, 8, 32, 3, 2, 1, 16),     # depthwise multiplier 2, stride 2
    (2, 32, 10, 10, 64, 3, 1, 1, 4),    # 8 -> 16 channels per group
    (1, 24, 11, 9, 24, 5, 1, 2, 3),     # 5x5, 8 channels per group
    (2, 128, 8, 8, 128, 3, 1, 1, 32),   # ResNeXt-style 4 channels per group
]


@pytest.mark.parametrize("case", GRAD_CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("layout", ["NHWC", "NCHW"])
@pytest.mark.parametrize("ind", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_grouped_gradients_match_oracle(case, layout, ind):
    N, C, H, W, K, R, st, pd, G = case
    if ind == torch.bfloat16 and layout == "NCHW":
        pytest.skip("BF16 gradients take NHWC")
    p = oracle.Conv(N, C, H, W, K, R, R, st, pd, 1, layout, groups=G)
    g = torch.Generator().manual_seed(97 + G)
    x = torch.randn(p.x_shape, generator=g).to(ind)
    w = (torch.randn(p.w_shape, generator=g) / np.sqrt(C // G * R * R)).to(ind)
    gy = torch.randn(p.y_shape, generator=g).to(ind)
    dx = F.conv2d_dgrad(gy.cuda(), w.cuda(), tuple(x.shape), st, pd, 1, layout,
                        out_dtype=torch.float32, groups=G)
    dw, db = F.conv2d_wgrad(x.cuda(), gy.cuda(), tuple(w.shape), st, pd, 1, layout, groups=G)
    F.device_error()
    dxr, dxb = oracle.conv2d_dgrad(p, f64(gy), f64(w), with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(x), f64(gy), with_bound=True)
    dbr, dbb = oracle.conv2d_bgrad(p, f64(gy), with_bound=True)
    tol = TOL_F32 if ind == torch.float32 else TOL_ACC32
    assert oracle.max_normalised_error(f64(dx), dxr, dxb) <= tol
    assert oracle.max_normalised_error(f64(dw), dwr, dwb) <= tol
    assert oracle.max_normalised_error(f64(db), dbr, dbb) <= tol


def test_grouped_autograd_relu_matches_oracle():
    """Depthwise layer with ReLU through Conv2dFn (the library masks the
    gradient, then the grouped data and weight gradients)."""
    N, C, H, W, G = 2, 16, 8, 8, 16
    p = oracle.Conv(N, C, H, W, C, 3, 3, 1, 1, 1, "NHWC", groups=G)
    g = torch.Generator().manual_seed(99)
    x = torch.randint(-3, 4, p.x_shape, generator=g).float()
    w = torch.randint(-3, 4, p.w_shape, generator=g).float()
    b = torch.randint(-4, 4, (C,), generator=g).float() + 0.5
    gy = torch.randn(p.y_shape, generator=g)
    xg, wg, bg = (t.cuda().requires_grad_() for t in (x, w, b))
    y = F.conv2d_autograd(xg, wg, bg, 1, 1, 1, True, "NHWC", groups=G)
    y.backward(gy.cuda())
    F.device_error()
    z = oracle.conv2d_fwd(p, f64(x), f64(w), f64(b))
    assert np.min(np.abs(z)) >= 0.5
    gz = oracle.relu_grad(np.maximum(z, 0.0), f64(gy))
    dxr, dxb = oracle.conv2d_dgrad(p, gz, f64(w), with_bound=True)
    dwr, dwb = oracle.conv2d_wgrad(p, f64(x), gz, with_bound=True)
    assert oracle.max_normalised_error(f64(xg.grad), dxr, dxb) <= TOL_F32
    assert oracle.max_normalised_error(f64(wg.grad), dwr, dwb) <= TOL_F32
