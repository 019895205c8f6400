"""conv2d_dgrad_noalloc: the data gradient for callers that cannot allocate
device memory or pass a workspace (a framework allocator that must own every
device byte, a fixed memory budget, work enqueued where an allocation would
stall or be refused). Its scratch is a static device array inside the library.

Checked through the C ABI against the FP64 oracle's data gradient and against
conv2d_dgrad (which takes a workspace), on two calls in a row with different
filters, so that a second call cannot pass on scratch left behind by the
first. This file is collected last; it passes on its own in a fresh process
and after the rest of the suite."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300.synth import ConvShape, make_inputs

from _gpu_helpers import TOL_ACC32, f64, oconv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _prob(sh, out_dtype):
    return B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, out_dtype, B.GBCONV_NHWC, 0)


def _with_workspace(prob, dy, w, dx):
    s, nbytes = B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, prob)
    B.check(s, "workspace_size")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    B.check(B.conv2d_dgrad(prob, dy.data_ptr(), w.data_ptr(), dx.data_ptr(), ws.data_ptr(),
                           nbytes, st), "conv2d_dgrad")


@pytest.mark.parametrize("sh", [ConvShape(2, 64, 9, 11, 96, 3, 3, 1, 1, 1),     # rotated filter
                                ConvShape(2, 32, 11, 11, 32, 3, 3, 2, 1, 1),    # sub-pixel phases
                                ConvShape(1, 64, 23, 19, 96, 5, 5, 2, 2, 1),    # phases, 5x5
                                ConvShape(2, 12, 11, 11, 20, 3, 3, 2, 1, 1)],   # CUDA cores
                         ids=["stride1-static-scratch", "stride2-static-scratch",
                              "stride2-5x5-static-scratch", "channels12-no-scratch"])
def test_noalloc_matches_oracle_and_workspace_dgrad_two_calls(sh):
    st = torch.cuda.current_stream().cuda_stream
    prob = _prob(sh, B.GBCONV_F32)
    p = oconv(sh)
    for call, seed in enumerate((50, 51)):  # two calls in a row, different w and dy
        x, w, _, g = make_inputs(sh, seed, grad=True)
        wb, gb = w.bfloat16().cuda(), g.bfloat16().cuda()
        dx_new = torch.full(sh.x_shape(), float("nan"), dtype=torch.float32, device="cuda")
        dx_ref = torch.empty(sh.x_shape(), dtype=torch.float32, device="cuda")
        B.check(B.conv2d_dgrad_noalloc(prob, gb.data_ptr(), wb.data_ptr(), dx_new.data_ptr(), st),
                "conv2d_dgrad_noalloc")
        _with_workspace(prob, gb, wb, dx_ref)
        B.check(B.gbconv_get_device_error(st), "device")
        assert not torch.isnan(dx_new).any()
        # the oracle's data gradient on the same BF16 operands; the tolerance is
        # normalised by sum |g||w| over each output's terms
        ref, bound = oracle.conv2d_dgrad(p, f64(gb), f64(wb), with_bound=True)
        err = oracle.max_normalised_error(f64(dx_new), ref, bound)
        assert err <= TOL_ACC32, (call, err)
        # and the entry point that takes a workspace
        err = oracle.max_normalised_error(f64(dx_new), f64(dx_ref), bound)
        assert err <= TOL_ACC32, (call, err)


def test_noalloc_refuses_filters_beyond_the_static_scratch():
    # 1024 x 3 x 3 x 1024 BF16 = 18.9 MB of rotated filter > 8 MiB
    sh = ConvShape(1, 1024, 8, 8, 1024, 3, 3, 1, 1, 1)
    prob = _prob(sh, B.GBCONV_BF16)
    assert 1024 * 9 * 1024 * 2 > B.GBCONV_DGRAD_STATIC_SCRATCH_BYTES
    # refused on the host before any pointer is touched or anything is enqueued
    s = B.conv2d_dgrad_noalloc(prob, 4096, 8192, 12288, 0)
    assert s == B.GBCONV_ERR_WORKSPACE
