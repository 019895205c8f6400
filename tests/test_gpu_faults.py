"""Failure detection without a GPU fault: the test control
GBCONV_DEBUG_SKIP_LOADS makes the tensor-core producer (and the staged
depthwise kernel's copy issuer) issue no loads, so the consumers' bounded
waits run out; the kernel must record a timeout, free its Tensor Memory and
return, and the context must stay usable."""
import pytest
import torch

from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, make_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("sh", [ConvShape(2, 64, 9, 9, 64, 3, 3, 1, 1, 1),      # one SM per tile
                                ConvShape(3, 128, 9, 9, 128, 3, 3, 1, 1, 1),    # SM pairs
                                ConvShape(2, 64, 9, 9, 256, 3, 3, 1, 1, 1)],    # 256 channels
                         ids=["pband", "pband-pair", "k256"])
def test_wait_timeout_reported_and_context_survives(sh):
    x, w, b, _ = make_inputs(sh, 40)
    xb, wb, bb = x.bfloat16().cuda(), w.bfloat16().cuda(), b.cuda()
    ref = F.conv2d(xb, wb, bb, 1, 1, 1, True)
    F.device_error()
    B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 20_000_000), "debug")  # 20 ms
    B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 1), "debug")
    try:
        F.conv2d(xb, wb, bb, 1, 1, 1, True)
        # every CTA gives up on its first wait: the call ends within the limits
        st = B.gbconv_get_device_error(torch.cuda.current_stream().cuda_stream)
        assert st == B.GBCONV_ERR_TIMEOUT
    finally:
        B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 0)
        B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 0)
    # the word was cleared and the next launch (which needs all TMEM) works
    y = F.conv2d(xb, wb, bb, 1, 1, 1, True)
    F.device_error()
    assert torch.equal(y, ref)


def test_staged_depthwise_wait_timeout_reported():
    """The staged depthwise kernel waits on its row copies with the same
    bounded wait: no copies issued -> timeout recorded, context usable."""
    N, C, H, W = 2, 64, 9, 9
    g = torch.Generator().manual_seed(41)
    xb = torch.randn(N, H, W, C, generator=g).bfloat16().cuda()
    wb = (torch.randn(C, 3, 3, 1, generator=g) / 3).bfloat16().cuda()
    ref = F.conv2d(xb, wb, None, 1, 1, 1, True, groups=C)
    F.device_error()
    B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 20_000_000), "debug")  # 20 ms
    B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 1), "debug")
    try:
        F.conv2d(xb, wb, None, 1, 1, 1, True, groups=C)
        st = B.gbconv_get_device_error(torch.cuda.current_stream().cuda_stream)
        assert st == B.GBCONV_ERR_TIMEOUT
    finally:
        B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 0)
        B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 0)
    y = F.conv2d(xb, wb, None, 1, 1, 1, True, groups=C)
    F.device_error()
    assert torch.equal(y, ref)


@pytest.mark.parametrize("algo", ["im2col", "band"])
def test_wgrad_wait_timeout_reported(algo):
    """Both tensor-core weight-gradient kernels: no loads issued -> the MMA
    and epilogue waits run out, the timeout is recorded, TMEM is freed, and
    the next call gives the same gradients as before."""
    sh = ConvShape(2, 64, 9, 9, 64, 3, 3, 1, 1, 1)
    x, w, _, g = make_inputs(sh, 42, grad=True)
    xb, gb = x.bfloat16().cuda(), g.bfloat16().cuda()
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, 1, 1, 1, B.GBCONV_BF16,
                     B.GBCONV_BF16)
    a = B.GBCONV_ALGO_SHIFT if algo == "band" else B.GBCONV_ALGO_IM2COL
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob, B.gbconv_config_t(0, 0, 4, 0, a)),
            "set_config")
    try:
        ref = F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
        F.device_error()
        B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 20_000_000), "debug")  # 20 ms
        B.check(B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 1), "debug")
        try:
            F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
            st = B.gbconv_get_device_error(torch.cuda.current_stream().cuda_stream)
            assert st == B.GBCONV_ERR_TIMEOUT
        finally:
            B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 0)
            B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 0)
        dw, db = F.conv2d_wgrad(xb, gb, tuple(w.shape), 1, 1, 1)
        F.device_error()
        assert torch.equal(dw, ref[0]) and torch.equal(db, ref[1])
    finally:
        B.gbconv_shutdown()
