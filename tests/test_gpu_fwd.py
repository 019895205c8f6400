"""GPU parity of the forward convolution (CUDA-core FP32 kernel, tcgen05 BF16
and FP8 kernels) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import (ConvShape, config_fp8, config_tiny_fp32, make_inputs,
                                          resnet_layers)

from _gpu_helpers import (TOL_ACC32, TOL_BF16, TOL_BF16_OUT, TOL_F32, TOL_FP8, f64, fp8_case,
                          fwd_case, oconv, set_block_n)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    yield
    B.gbconv_shutdown()


# ---------------- plain FP32 kernel ----------------

def test_fp32_tiny_config():
    """FP32 NCHW N=1 C=3 32x32 K=16 3x3 pad 1 with bias, U[-1,1] from seed 0."""
    sh = config_tiny_fp32()
    r = fwd_case(sh, torch.float32, relu=False, seed=0, x_dist="uniform", w_dist="uniform")
    assert r["err_i"] <= TOL_F32, r["err_i"]


FP32_SHAPES = [
    ConvShape(2, 5, 9, 11, 7, 3, 3, 1, 1, 1, "NCHW"),
    ConvShape(2, 5, 9, 11, 7, 3, 3, 1, 1, 1, "NHWC"),
    ConvShape(3, 17, 13, 12, 70, 3, 3, 2, 1, 1, "NHWC"),
    ConvShape(3, 17, 13, 12, 70, 3, 3, 2, 1, 1, "NCHW"),
    ConvShape(1, 8, 15, 15, 9, 3, 3, 1, 2, 2, "NHWC"),
    ConvShape(2, 4, 10, 10, 3, 5, 3, (2, 1), (2, 0), (1, 2), "NCHW"),
    ConvShape(2, 33, 7, 7, 130, 1, 1, 1, 0, 1, "NHWC"),
    ConvShape(1, 3, 20, 20, 5, 7, 7, 2, 3, 1, "NCHW"),
]


@pytest.mark.parametrize("sh", FP32_SHAPES, ids=lambda s: f"{s.layout}-{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}-s{s.stride}-d{s.dil}")
@pytest.mark.parametrize("relu", [False, True])
def test_fp32_shapes(sh, relu):
    r = fwd_case(sh, torch.float32, relu=relu, seed=3, x_dist="uniform", w_dist="uniform")
    assert r["err_i"] <= TOL_F32


def test_fp32_integer_exact():
    sh = ConvShape(2, 9, 11, 10, 13, 3, 3, 1, 1, 1, "NCHW")
    r = fwd_case(sh, torch.float32, relu=False, seed=4, x_dist=("int", -4, 4),
                 w_dist=("int", -4, 4))
    assert np.array_equal(r["got"], r["ref"].reshape(-1))


def test_fp32_empty_batch():
    sh = ConvShape(0, 4, 8, 8, 4, 3, 3, 1, 1, 1, "NCHW")
    x = torch.zeros(0, 4, 8, 8, device="cuda")
    w = torch.zeros(4, 4, 3, 3, device="cuda")
    y = F.conv2d(x, w, None, 1, 1, 1, False, "NCHW")
    F.device_error()
    assert y.shape == (0, 4, 8, 8)


# ---------------- BF16 tensor-core kernel ----------------

BF16_SHAPES = [
    ConvShape(2, 64, 8, 8, 64, 1, 1, 1, 0, 1),       # one channel block, 1x1
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),      # ragged pixel tail
    ConvShape(3, 128, 12, 12, 128, 3, 3, 2, 1, 1),   # stride 2
    ConvShape(1, 16, 15, 13, 48, 3, 3, 1, 2, 2),     # dilation 2, C < 64, K not /32
    ConvShape(2, 72, 10, 10, 40, 5, 5, 1, 2, 1),     # partial channel block, partial n tile
    ConvShape(1, 32, 21, 21, 64, 7, 7, 2, 3, 1),     # 7x7 stride 2 (stem-like)
    ConvShape(2, 256, 7, 7, 256, 3, 3, 1, 1, 1),
    ConvShape(2, 24, 9, 9, 24, 3, 1, (1, 2), (1, 0), 1),  # rectangular filter, per-axis stride
    ConvShape(4, 64, 14, 14, 512, 1, 1, 2, 0, 1),    # 1x1 stride-2 downsample
]


def _id(s):
    return f"{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}x{s.S}-s{s.stride}-p{s.pad}-d{s.dil}"


@pytest.mark.parametrize("sh", BF16_SHAPES, ids=_id)
def test_bf16_shapes_bf16_out(sh):
    r = fwd_case(sh, torch.bfloat16, relu=True, seed=5)
    assert r["err_i"] <= TOL_BF16_OUT, r["err_i"]
    assert r["err_ii"] <= TOL_BF16, r["err_ii"]


@pytest.mark.parametrize("sh", BF16_SHAPES, ids=_id)
def test_bf16_shapes_f32_out(sh):
    r = fwd_case(sh, torch.bfloat16, out_dtype=torch.float32, relu=False, seed=6)
    assert r["err_i"] <= TOL_ACC32, r["err_i"]


@pytest.mark.parametrize("block_n", [32, 64, 128, 256])
@pytest.mark.parametrize("raster", [0, 1])
def test_bf16_every_tile_width(block_n, raster):
    sh = ConvShape(2, 64, 13, 13, 256, 3, 3, 1, 1, 1)
    set_block_n(sh, B.GBCONV_BF16, B.GBCONV_F32, block_n, raster=raster)
    try:
        r = fwd_case(sh, torch.bfloat16, out_dtype=torch.float32, relu=False, bias=False, seed=7)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= TOL_ACC32


@pytest.mark.parametrize("sh", [ConvShape(2, 16, 9, 9, 24, 3, 3, 1, 1, 1),
                                ConvShape(3, 64, 11, 7, 136, 3, 3, 2, 1, 1),
                                ConvShape(1, 8, 12, 12, 8, 5, 5, 1, 4, 2)], ids=_id)
def test_bf16_integer_exact(sh):
    """x, w in {-4..4}, b in {-8..8}: every partial sum is an integer below
    2^24, so FP32 accumulation is exact: FP32 output must equal the oracle
    bit for bit, BF16 output too wherever |y| <= 256."""
    r = fwd_case(sh, torch.bfloat16, out_dtype=torch.float32, relu=False, seed=8,
                 x_dist=("int", -4, 4), w_dist=("int", -4, 4))
    assert np.array_equal(r["got"], r["ref"].reshape(-1))
    r = fwd_case(sh, torch.bfloat16, relu=False, seed=8, x_dist=("int", -4, 4),
                 w_dist=("int", -4, 4))
    ref = r["ref"].reshape(-1)
    small = np.abs(ref) <= 256
    assert small.mean() > 0.5
    assert np.array_equal(r["got"][small], ref[small])


def test_bf16_identity_and_shift():
    """1x1 identity filter reproduces x; a delta filter shifts it (exactly)."""
    dev = "cuda"
    sh = ConvShape(2, 64, 9, 10, 64, 3, 3, 1, 1, 1)
    x, _, _, _ = make_inputs(sh, 9, bias=False)
    xb = x.bfloat16().to(dev)
    eye = torch.zeros(64, 1, 1, 64)
    eye[torch.arange(64), 0, 0, torch.arange(64)] = 1
    y = F.conv2d(xb, eye.bfloat16().to(dev), None, 1, 0, 1, False, "NHWC")
    F.device_error()
    assert torch.equal(y.cpu(), xb.cpu())
    delta = torch.zeros(64, 3, 3, 64)
    delta[torch.arange(64), 2, 0, torch.arange(64)] = 1   # tap (r, s) = (2, 0)
    y = F.conv2d(xb, delta.bfloat16().to(dev), None, 1, 1, 1, False, "NHWC").cpu()
    F.device_error()
    # y[n,p,q,c] = x[n, p + 2 - 1, q + 0 - 1, c]
    exp = torch.zeros_like(y)
    exp[:, 0:8, 1:10, :] = xb.cpu()[:, 1:9, 0:9, :]
    assert torch.equal(y, exp)


def test_bf16_deterministic_and_guarded():
    """Two runs are bitwise equal, and nothing outside y is written."""
    sh = ConvShape(3, 64, 13, 13, 96, 3, 3, 1, 1, 1)
    x, w, b, _ = make_inputs(sh, 10)
    dev = "cuda"
    xb, wb, bb = x.bfloat16().to(dev), w.bfloat16().to(dev), b.to(dev)
    n = int(np.prod(sh.y_shape()))
    guard = 4096
    buf = torch.full((n + 2 * guard,), 7.0, dtype=torch.bfloat16, device=dev)
    y1 = buf[guard:guard + n].view(sh.y_shape())
    F.conv2d(xb, wb, bb, 1, 1, 1, True, "NHWC", out=y1)
    first = y1.clone()
    F.conv2d(xb, wb, bb, 1, 1, 1, True, "NHWC", out=y1)
    F.device_error()
    assert torch.equal(first, y1)
    assert torch.all(buf[:guard] == 7.0) and torch.all(buf[guard + n:] == 7.0)


def test_bf16_empty_batch():
    x = torch.zeros(0, 8, 8, 64, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(64, 3, 3, 64, dtype=torch.bfloat16, device="cuda")
    y = F.conv2d(x, w, None, 1, 1, 1, False, "NHWC")
    F.device_error()
    assert y.shape == (0, 8, 8, 64)


@pytest.mark.parametrize("li", range(4))
def test_resnet_layer_full_size_every_output(li):
    """The ResNet bottleneck layers at batch 32, in the configuration the bench
    times (BF16 in/out, bias + ReLU): every output against the oracle."""
    sh = resnet_layers()[li]
    r = fwd_case(sh, torch.bfloat16, relu=True, seed=20 + li)
    assert r["err_i"] <= TOL_BF16_OUT, r["err_i"]
    assert r["err_ii"] <= TOL_BF16, r["err_ii"]


@pytest.mark.parametrize("li", range(4))
def test_resnet_layer_fp32_kernel_every_output(li):
    """The plain FP32 kernel on the same layers (NHWC FP32), every output."""
    sh = resnet_layers()[li]
    r = fwd_case(sh, torch.float32, relu=True, seed=20 + li)
    assert r["err_i"] <= TOL_F32, r["err_i"]


# ---------------- FP8 E4M3 ----------------

def test_quantize_e4m3_matches_oracle():
    """GPU operand preparation: scale = max|v|/448 and RNE-saturating E4M3
    codes, bit for bit the oracle's (both in binary32)."""
    torch.manual_seed(0)
    for rows, shape in [(1, (4, 7, 9, 32)), (16, (16, 3, 3, 48))]:
        t = torch.randn(shape) * 3
        t.view(-1)[5] = 0.0
        q, s = F.quantize_e4m3(t.cuda(), rows=rows)
        codes, scales = oracle.scale_quant_e4m3(t.numpy(), rows)
        assert np.array_equal(s.cpu().numpy(), scales)
        got = q.view(torch.uint8).cpu().numpy()
        # -0 and +0 both decode to zero; compare values, then codes elsewhere
        assert np.array_equal(oracle.e4m3_to_f64(got), oracle.e4m3_to_f64(codes))
        nz = oracle.e4m3_to_f64(codes) != 0
        assert np.array_equal(got[nz], codes[nz])
    # bf16 input path
    tb = (torch.randn(2, 5, 5, 64) * 0.1).bfloat16()
    q, s = F.quantize_e4m3(tb.cuda(), rows=1)
    codes, scales = oracle.scale_quant_e4m3(tb.float().numpy(), 1)
    assert np.array_equal(s.cpu().numpy(), scales)
    assert np.array_equal(oracle.e4m3_to_f64(q.view(torch.uint8).cpu().numpy()),
                          oracle.e4m3_to_f64(codes))


@pytest.mark.parametrize("n", [64 * 28 * 28 * 256, 100003, 1 << 16])
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_quantize_e4m3_large_tensor_matches_oracle(n, dt):
    """Per-tensor preparation of large tensors (the FP8 workload's activation,
    and lengths that are not a multiple of the 8-value vector): scale and
    every code bit for bit the oracle's."""
    g = torch.Generator().manual_seed(n % 997)
    t = (torch.randn(n, generator=g) * 2).clamp_min(0).to(dt)
    t[7] = -5.0  # the largest magnitude may be negative
    q, sc = F.quantize_e4m3(t.cuda(), rows=1)
    F.device_error()
    codes, scales = oracle.scale_quant_e4m3(t.float().numpy(), 1)
    assert np.array_equal(sc.cpu().numpy(), scales)
    got = q.view(torch.uint8).cpu().numpy()
    assert np.array_equal(oracle.e4m3_to_f64(got), oracle.e4m3_to_f64(codes))
    nz = oracle.e4m3_to_f64(codes) != 0
    assert np.array_equal(got[nz], codes[nz])


def _e4m3_midpoints():
    """Every midpoint between consecutive non-negative E4M3 values up to 448."""
    vals = np.unique(np.abs(oracle.e4m3_to_f64(np.arange(256, dtype=np.uint8))))
    vals = vals[np.isfinite(vals) & (vals <= 448)]
    return (vals[:-1] + vals[1:]) / 2


@pytest.mark.parametrize("length", [4096, 4093], ids=["vector", "scalar"])
def test_quantize_e4m3_near_rounding_midpoints(length):
    """Quotients v/s at and within three binary32 steps of every E4M3
    rounding midpoint, both signs, eight rows with their own scales: the
    GPU's binary32 quotient and E4M3 code equal the oracle's for each (the
    ties of either rounding are where a wrong quotient would show)."""
    rng = np.random.default_rng(11)
    mids = _e4m3_midpoints().astype(np.float32)
    rows = 8
    t = np.zeros((rows, length), dtype=np.float32)
    for r in range(rows):
        amax = np.float32(rng.uniform(0.5, 4.0) * 10.0 ** rng.integers(-3, 4))
        s = np.float32(amax / np.float32(448.0))
        vals = [amax]
        for m in mids:
            v = np.float32(m * s)
            for k in range(-3, 4):
                w = v
                for _ in range(abs(k)):
                    w = np.nextafter(w, np.float32(np.inf if k > 0 else -np.inf), dtype=np.float32)
                if abs(w) <= amax:
                    vals += [w, -w]
        vals = np.array(vals, dtype=np.float32)
        assert len(vals) <= length
        t[r, :len(vals)] = vals
    q, sc = F.quantize_e4m3(torch.from_numpy(t).cuda(), rows=rows)
    F.device_error()
    codes, scales = oracle.scale_quant_e4m3(t, rows)
    assert np.array_equal(sc.cpu().numpy(), scales)
    got = q.view(torch.uint8).cpu().numpy().reshape(-1)
    codes = codes.reshape(-1)
    assert np.array_equal(oracle.e4m3_to_f64(got), oracle.e4m3_to_f64(codes))
    nz = oracle.e4m3_to_f64(codes) != 0
    assert np.array_equal(got[nz], codes[nz])


@pytest.mark.parametrize("sh", [ConvShape(2, 32, 9, 9, 32, 3, 3, 1, 1, 1),
                                ConvShape(3, 128, 10, 10, 64, 3, 3, 1, 1, 1),
                                ConvShape(2, 144, 8, 8, 40, 1, 1, 1, 0, 1),
                                ConvShape(2, 64, 12, 12, 128, 3, 3, 2, 1, 1)], ids=_id)
def test_fp8_small(sh):
    r = fp8_case(sh, seed=11)
    assert r["err_i"] <= TOL_BF16_OUT, r["err_i"]
    assert r["err_ii"] <= TOL_FP8, r["err_ii"]


def test_fp8_full_size_every_output():
    """FP8 workload: N=64, C=K=256, 28x28, 3x3 pad 1, ReLU(N(0,1)) activations;
    every one of the 12.8 M outputs against the oracle."""
    sh = config_fp8()
    r = fp8_case(sh, seed=12)
    assert r["err_i"] <= TOL_BF16_OUT, r["err_i"]
    assert r["err_ii"] <= TOL_FP8, r["err_ii"]


# ---------------- both forward algorithms on the same layers ----------------

ALGO_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),
    ConvShape(1, 16, 15, 13, 48, 3, 3, 1, 2, 2),
    ConvShape(2, 72, 10, 10, 40, 5, 5, 1, 2, 1),
    ConvShape(2, 64, 30, 60, 96, 3, 3, 1, 1, 1),       # Wx = 64 ... 128 boundary (Q + 2 = 62)
    ConvShape(1, 64, 6, 100, 64, 3, 3, 1, 1, 1),       # Wx = 128 (Q + 2 = 102), one row per tile
    ConvShape(2, 32, 7, 7, 32, 1, 1, 1, 0, 1),         # 1x1 forced onto the band kernel
    ConvShape(3, 64, 9, 9, 64, 3, 5, 1, (1, 2), 1),    # rectangular filter
]


@pytest.mark.parametrize("sh", ALGO_SHAPES, ids=_id)
@pytest.mark.parametrize("algo", [B.GBCONV_ALGO_IM2COL, B.GBCONV_ALGO_SHIFT, B.GBCONV_ALGO_SHIFT_T])
@pytest.mark.parametrize("block_n", [64, 128])
def test_bf16_forward_algorithms(sh, algo, block_n):
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, B.GBCONV_F32, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS)
    B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob,
                                B.gbconv_config_t(block_n, 0, 0, 0, algo)), "set_config")
    try:
        r = fwd_case(sh, torch.bfloat16, out_dtype=torch.float32, relu=False, seed=70)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= TOL_ACC32, r["err_i"]


T_SHAPES = [  # the transposed band kernel: K <= 128, both output-channel tiles
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),
    ConvShape(2, 64, 10, 10, 40, 3, 3, 1, 1, 1),      # K < 64: clipped channels
    ConvShape(2, 128, 9, 9, 128, 3, 3, 1, 1, 1),      # two channel blocks, 128 channels
    ConvShape(1, 64, 12, 12, 96, 5, 5, 1, 2, 1),      # 96 channels on a 128 tile
    ConvShape(2, 32, 20, 30, 64, 3, 3, 1, 2, 2),      # dilation 2
    ConvShape(1, 64, 5, 120, 64, 3, 3, 1, 1, 1),      # Wx = 128, two rows per tile
    ConvShape(1, 64, 4, 150, 32, 1, 3, 1, (0, 1), 1),  # Wx = 256, one row per tile
    # strided layers: taps grouped into phase images, one strided band per phase
    ConvShape(2, 128, 17, 15, 128, 3, 3, 2, 1, 1),    # 4 phases (4, 2, 2, 1 taps), ragged
    ConvShape(2, 64, 20, 22, 64, 3, 3, 2, 1, 1),
    ConvShape(1, 64, 23, 19, 96, 5, 5, 2, 2, 1),      # shifts 0..2 in each phase
    ConvShape(1, 32, 16, 40, 48, 3, 3, (2, 1), 1, 1),  # row stride only: 2 phases
    ConvShape(1, 64, 22, 25, 64, 7, 7, 2, 3, 1),      # 7x7 stride 2, streamed filter
    ConvShape(1, 64, 21, 21, 64, 3, 3, 2, 2, 2),      # stride 2, dilation 2: one phase
    ConvShape(1, 64, 25, 25, 64, 3, 3, 3, 1, 1),      # stride 3: a phase per tap
    ConvShape(1, 64, 9, 180, 64, 3, 3, 2, 1, 1),      # Wx = 128 at column stride 2
    # 1x1 stride-1 layers: flat GEMM over N*H*W positions, ragged last tile
    ConvShape(3, 64, 7, 9, 64, 1, 1, 1, 0, 1),        # 189 positions: one partial tile
    ConvShape(2, 128, 15, 17, 256, 1, 1, 1, 0, 1),    # 256 channels: two channel tiles
    ConvShape(1, 256, 20, 21, 96, 1, 1, 1, 0, 1),     # four channel blocks, K on a 128 tile
]


@pytest.mark.parametrize("sh", T_SHAPES, ids=_id)
@pytest.mark.parametrize("out", ["bf16", "f32"])
def test_bf16_transposed_band_kernel(sh, out):
    od = B.GBCONV_F32 if out == "f32" else B.GBCONV_BF16
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, od, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU)
    B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob,
                                B.gbconv_config_t(64, 0, 0, 0, B.GBCONV_ALGO_SHIFT_T)), "set_config")
    try:
        r = fwd_case(sh, torch.bfloat16, out_dtype=torch.float32 if out == "f32" else None,
                     relu=True, seed=72)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= (TOL_ACC32 if out == "f32" else TOL_BF16_OUT), r["err_i"]


@pytest.mark.parametrize("algo", [B.GBCONV_ALGO_IM2COL, B.GBCONV_ALGO_SHIFT_T])
@pytest.mark.parametrize("sh", [ConvShape(2, 256, 19, 17, 128, 3, 3, 2, 1, 1),
                                ConvShape(2, 256, 13, 19, 192, 1, 1, 1, 0, 1)], ids=_id)
def test_fp8_strided_and_flat_forward(algo, sh):
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_E4M3, B.GBCONV_BF16, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS)
    B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob, B.gbconv_config_t(128, 0, 0, 0, algo)),
            "set_config")
    try:
        r = fp8_case(sh, seed=73)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= TOL_BF16_OUT and r["err_ii"] <= TOL_FP8, r


@pytest.mark.parametrize("algo", [B.GBCONV_ALGO_IM2COL, B.GBCONV_ALGO_SHIFT])
def test_fp8_forward_algorithms(algo):
    sh = ConvShape(2, 256, 12, 12, 128, 3, 3, 1, 1, 1)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_E4M3,
                     B.GBCONV_BF16, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS)
    B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob, B.gbconv_config_t(128, 0, 0, 0, algo)),
            "set_config")
    try:
        r = fp8_case(sh, seed=71)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= TOL_BF16_OUT and r["err_ii"] <= TOL_FP8, r


# ---------------- the FP32 NHWC fast path (C, K multiples of 4) ----------------

FAST_F32_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),        # ragged pixel tile, 64-column tile
    ConvShape(1, 4, 7, 7, 4, 3, 3, 1, 1, 1),           # one channel vector, one output vector
    ConvShape(2, 20, 10, 10, 68, 3, 3, 1, 1, 1),       # partial channel block, K past 64
    ConvShape(2, 128, 12, 12, 128, 3, 3, 2, 1, 1),     # stride 2, 128-column tile
    ConvShape(1, 64, 15, 13, 200, 3, 3, 1, 2, 2),      # dilation 2, two 128-column tiles
    ConvShape(3, 256, 7, 7, 64, 1, 1, 1, 0, 1),        # 1x1
    ConvShape(1, 32, 9, 16, 48, 5, 3, (2, 1), (2, 1), 1),  # rectangular filter, row stride
]


@pytest.mark.parametrize("sh", FAST_F32_SHAPES, ids=_id)
def test_fp32_fast_path_matches_oracle(sh):
    r = fwd_case(sh, torch.float32, relu=True, seed=160)
    assert r["err_i"] <= TOL_F32, r["err_i"]


def test_fp32_fast_path_integer_exact():
    """Integer operands: every partial sum is exact in FP32, so the register-
    blocked FFMA kernel equals the oracle bit for bit."""
    sh = ConvShape(2, 64, 11, 10, 96, 3, 3, 1, 1, 1)
    x, w, b, _ = make_inputs(sh, 161, x_dist=("int", -4, 4), w_dist=("int", -4, 4))
    y = F.conv2d(x.cuda(), w.cuda(), b.cuda(), 1, 1, 1, False, "NHWC")
    F.device_error()
    ref = oracle.conv2d_fwd(oconv(sh), f64(x), f64(w), f64(b))
    assert np.array_equal(f64(y), ref)


def test_fp32_fast_path_fused_residual_in_place():
    sh = ConvShape(2, 32, 8, 9, 64, 3, 3, 1, 1, 1)
    x, w, b, _ = make_inputs(sh, 162)
    g = torch.Generator().manual_seed(163)
    alpha = torch.rand(sh.K, generator=g) + 0.5
    z = torch.randn(sh.y_shape(), generator=g)
    yz = z.clone().cuda()
    F.conv2d_fused(x.cuda(), w.cuda(), b.cuda(), alpha.cuda(), yz, 1, 1, 1, True, out=yz)
    F.device_error()
    ref, bound = oracle.conv2d_fwd_fused(oconv(sh), f64(x), f64(w), f64(alpha), f64(b), f64(z),
                                          relu=True, with_bound=True)
    assert oracle.max_normalised_error(f64(yz), ref, bound) <= TOL_F32
