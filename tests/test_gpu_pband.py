"""GPU parity of the pixel-major band kernel (GBCONV_ALGO_PBAND: one SM per
128-position tile; GBCONV_ALGO_PBAND_PAIR: two SMs per 256-row MMA, each
holding half of the filter), against the FP64 oracle: ragged tiles, output
channels below a tile, several channel blocks, dilation, strides 2 and 3 by
phases, rectangular filters, BF16 and FP32 outputs, and integer operands for
which the FP32 result must equal the oracle bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, make_inputs, resnet_layers

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, f64, fwd_case, oconv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _id(s):
    return f"{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}x{s.S}-s{s.stride}-p{s.pad}-d{s.dil}"


P_SHAPES = [
    ConvShape(2, 64, 9, 11, 64, 3, 3, 1, 1, 1),           # ragged rows and columns
    ConvShape(2, 64, 10, 10, 40, 3, 3, 1, 1, 1),          # 40 channels on a 64 tile
    ConvShape(2, 128, 9, 9, 128, 3, 3, 1, 1, 1),          # two channel blocks, 128 channels
    ConvShape(1, 64, 12, 12, 96, 5, 5, 1, 2, 1),          # 96 channels on a 128 tile
    ConvShape(2, 32, 20, 30, 64, 3, 3, 1, 2, 2),          # dilation 2, a partial channel block
    ConvShape(1, 64, 5, 120, 64, 3, 3, 1, 1, 1),          # Wx = 122: one row per tile
    ConvShape(3, 256, 9, 9, 64, 3, 3, 1, 1, 1),           # four channel blocks
    ConvShape(3, 64, 13, 13, 128, 3, 1, 1, (1, 0), 1),    # 3x1 filter
    ConvShape(2, 128, 17, 15, 128, 3, 3, 2, 1, 1),        # stride 2: 4 phases (4, 2, 2, 1 taps)
    ConvShape(2, 64, 20, 22, 64, 3, 3, 2, 1, 1),
    ConvShape(1, 64, 23, 19, 96, 5, 5, 2, 2, 1),          # shifts 0..2 in each phase
    ConvShape(1, 32, 16, 40, 48, 3, 3, (2, 1), 1, 1),     # row stride only: 2 phases
    ConvShape(1, 64, 21, 21, 64, 3, 3, 2, 2, 2),          # stride 2, dilation 2: one phase
    ConvShape(1, 64, 25, 25, 64, 3, 3, 3, 1, 1),          # stride 3: a phase per tap
    ConvShape(5, 64, 7, 7, 64, 3, 3, 1, 1, 1),            # odd tile count: a pair's last half idles
]

ALGOS = {"one_sm": B.GBCONV_ALGO_PBAND, "pair": B.GBCONV_ALGO_PBAND_PAIR}


def _set(sh, algo, out_dtype, flags):
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, out_dtype, B.GBCONV_NHWC, flags)
    B.check(B.gbconv_set_config(B.GBCONV_OP_FWD, prob, B.gbconv_config_t(64, 0, 0, 0, algo)),
            "set_config")
    return prob


def _run_or_skip(fn):
    try:
        return fn()
    except B.GbconvError as e:
        if e.status == B.GBCONV_ERR_UNSUPPORTED:
            pytest.skip("this form cannot hold the layer's filter beside two band stages")
        raise


@pytest.mark.parametrize("sh", P_SHAPES, ids=_id)
@pytest.mark.parametrize("form", list(ALGOS), ids=list(ALGOS))
@pytest.mark.parametrize("out", ["bf16", "f32"])
def test_pband_matches_oracle(sh, form, out):
    od = B.GBCONV_F32 if out == "f32" else B.GBCONV_BF16
    _set(sh, ALGOS[form], od, B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU)
    try:
        r = _run_or_skip(lambda: fwd_case(sh, torch.bfloat16,
                                          out_dtype=torch.float32 if out == "f32" else None,
                                          relu=True, seed=140))
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= (TOL_ACC32 if out == "f32" else TOL_BF16_OUT), r["err_i"]


@pytest.mark.parametrize("sh", [P_SHAPES[0], P_SHAPES[2], P_SHAPES[8], P_SHAPES[13]], ids=_id)
@pytest.mark.parametrize("form", list(ALGOS), ids=list(ALGOS))
def test_pband_integer_exact(sh, form):
    """Integer x, w in [-4, 4] and b in [-8, 8]: every partial sum is an integer
    below 2^24, so the FP32 output equals the oracle bit for bit."""
    _set(sh, ALGOS[form], B.GBCONV_F32, B.GBCONV_FLAG_BIAS)
    x, w, b, _ = make_inputs(sh, 141, x_dist=("int", -4, 4), w_dist=("int", -4, 4))
    try:
        y = _run_or_skip(lambda: F.conv2d(x.bfloat16().cuda(), w.bfloat16().cuda(), b.cuda(),
                                          sh.stride, sh.pad, sh.dil, False, "NHWC", torch.float32))
        F.device_error()
    finally:
        B.gbconv_shutdown()
    ref = oracle.conv2d_fwd(oconv(sh), f64(x), f64(w), f64(b))
    assert np.array_equal(f64(y), ref)


def test_pband_repeatable_bitwise():
    """Two runs of the pair form give identical bits (fixed MMA order)."""
    sh = P_SHAPES[8]
    _set(sh, B.GBCONV_ALGO_PBAND_PAIR, B.GBCONV_BF16, B.GBCONV_FLAG_BIAS)
    x, w, b, _ = make_inputs(sh, 142)
    try:
        ys = [F.conv2d(x.bfloat16().cuda(), w.bfloat16().cuda(), b.cuda(), sh.stride, sh.pad,
                       sh.dil, False) for _ in range(2)]
        F.device_error()
    finally:
        B.gbconv_shutdown()
    assert torch.equal(ys[0], ys[1])


@pytest.mark.parametrize("li", [1, 3])
def test_resnet_3x3_layers_full_size_every_output(li):
    """The 3x3 ResNet layers at batch 32 on this kernel (one SM per tile for 64
    channels, pairs for 128): every output against the oracle."""
    sh = resnet_layers(32)[li]
    algo = B.GBCONV_ALGO_PBAND if sh.K <= 64 else B.GBCONV_ALGO_PBAND_PAIR
    _set(sh, algo, B.GBCONV_BF16, B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU)
    try:
        r = fwd_case(sh, torch.bfloat16, relu=True, seed=144)
    finally:
        B.gbconv_shutdown()
    assert r["err_i"] <= TOL_BF16_OUT, r["err_i"]
