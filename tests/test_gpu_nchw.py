"""GPU parity of the BF16 NCHW forward (layout transforms around the NHWC
tensor-core path) against the FP64 oracle in NCHW."""
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, make_inputs

from _gpu_helpers import TOL_ACC32, TOL_BF16_OUT, f64, oconv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


SHAPES = [
    ConvShape(2, 16, 9, 11, 24, 3, 3, 1, 1, 1, "NCHW"),
    ConvShape(2, 64, 14, 14, 128, 3, 3, 2, 1, 1, "NCHW"),
    ConvShape(1, 128, 7, 9, 256, 1, 1, 1, 0, 1, "NCHW"),
    ConvShape(2, 40, 13, 12, 72, 5, 3, 1, (2, 1), 1, "NCHW"),
]


def _id(s):
    return f"{s.N}x{s.C}x{s.H}x{s.W}-K{s.K}-R{s.R}x{s.S}-s{s.stride}"


@pytest.mark.parametrize("sh", SHAPES, ids=_id)
@pytest.mark.parametrize("out", ["bf16", "f32"])
@pytest.mark.parametrize("fused", [False, True])
def test_bf16_nchw_forward(sh, out, fused):
    od = torch.bfloat16 if out == "bf16" else torch.float32
    x, w, b, _ = make_inputs(sh, 95)
    xb, wb = x.bfloat16(), w.bfloat16()
    p = oconv(sh)
    g = torch.Generator().manual_seed(96)
    alpha = (torch.rand(sh.K, generator=g) + 0.5) if fused else None
    z = torch.randn(p.y_shape, generator=g).to(od) if fused else None
    dev = "cuda"
    if fused:
        y = F.conv2d_fused(xb.to(dev), wb.to(dev), b.to(dev), alpha.to(dev), z.to(dev), sh.stride,
                           sh.pad, sh.dil, True, "NCHW", out_dtype=od)
    else:
        y = F.conv2d(xb.to(dev), wb.to(dev), b.to(dev), sh.stride, sh.pad, sh.dil, True, "NCHW",
                     out_dtype=od)
    F.device_error()
    ref, bound = oracle.conv2d_fwd_fused(p, f64(xb), f64(wb), f64(alpha) if fused else None, f64(b),
                                         f64(z) if fused else None, relu=True, with_bound=True)
    err = oracle.max_normalised_error(f64(y).reshape(-1), ref.reshape(-1), bound.reshape(-1))
    assert err <= (TOL_BF16_OUT if out == "bf16" else TOL_ACC32), err
