"""The autotuner on the GPU: gbconv_tune times the candidate configurations of
the forward, data-gradient and weight-gradient kernels on the caller's
buffers, stores the fastest in the tuning table and returns it; the op then
runs with that configuration and must still match the FP64 oracle; the table
survives a save / clear / load round trip through its JSON file."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F
from paper_2207_00257_gb300.synth import ConvShape, make_inputs

from _gpu_helpers import TOL_ACC32, f64, oconv

pytestmark = pytest.mark.gpu

SHAPES = [ConvShape(2, 64, 14, 14, 64, 3, 3, 1, 1, 1),
          ConvShape(2, 128, 15, 13, 96, 3, 3, 2, 1, 1)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    yield
    B.gbconv_shutdown()


def _prob(sh):
    return B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, B.GBCONV_F32, B.GBCONV_NHWC, 0)


def _same(a, b):
    return (a.block_n, a.stages, a.split_k, a.raster, a.algo) == \
        (b.block_n, b.stages, b.split_k, b.raster, b.algo)


def _tune_and_run(op, sh, seed):
    x, w, _, g = make_inputs(sh, seed, grad=True)
    xb, wb, gb = x.bfloat16().cuda(), w.bfloat16().cuda(), g.bfloat16().cuda()
    prob = _prob(sh)
    st = torch.cuda.current_stream().cuda_stream
    s, nbytes = B.gbconv_workspace_size(op, prob)
    B.check(s, "workspace_size")
    # room for the widest weight-gradient split the tuner may try
    nbytes = max(nbytes, (64 * sh.K * sh.R * sh.S * sh.C + 128 * sh.K) * 4 + 256)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    if op == B.GBCONV_OP_FWD:
        out = torch.empty(sh.y_shape(), dtype=torch.float32, device="cuda")
        a, b = xb, wb
    elif op == B.GBCONV_OP_DGRAD:
        out = torch.empty(sh.x_shape(), dtype=torch.float32, device="cuda")
        a, b = gb, wb
    else:
        out = torch.empty(sh.w_shape(), dtype=torch.float32, device="cuda")
        a, b = xb, gb
    s, best = B.gbconv_tune(op, prob, a.data_ptr(), b.data_ptr(), 0, out.data_ptr(),
                            ws.data_ptr(), nbytes, 3, st)
    B.check(s, "gbconv_tune")
    s, stored = B.gbconv_get_config(op, prob)
    B.check(s, "get_config")
    assert _same(best, stored)
    # the stored config is one of the candidates the tuner tries
    if op == B.GBCONV_OP_WGRAD:
        assert best.split_k in (1, 2, 4, 8, 16, 32, 64)
    else:
        assert best.block_n in (0, 32, 64, 128, 256)
        if op == B.GBCONV_OP_DGRAD and sh.stride != (1, 1):
            # sub-pixel phases on the tensor cores, or the CUDA-core gather kernel
            assert best.algo in (B.GBCONV_ALGO_AUTO, B.GBCONV_ALGO_SIMT)
        else:
            assert best.algo in (B.GBCONV_ALGO_IM2COL, B.GBCONV_ALGO_SHIFT, B.GBCONV_ALGO_SHIFT_T,
                                 B.GBCONV_ALGO_PBAND, B.GBCONV_ALGO_PBAND_PAIR)
            assert best.stages in (0, 3, 4)
    # the op under the stored config, against the oracle
    p = oconv(sh)
    out.fill_(float("nan"))
    if op == B.GBCONV_OP_FWD:
        y = F.conv2d(xb, wb, None, sh.stride, sh.pad, sh.dil, False, "NHWC", torch.float32, out=out)
        F.device_error()
        ref, bound = oracle.conv2d_fwd(p, f64(xb), f64(wb), with_bound=True)
        err = oracle.max_normalised_error(f64(y), ref, bound)
    elif op == B.GBCONV_OP_DGRAD:
        dx = F.conv2d_dgrad(gb, wb, tuple(x.shape), sh.stride, sh.pad, sh.dil, "NHWC",
                            out_dtype=torch.float32)
        F.device_error()
        ref, bound = oracle.conv2d_dgrad(p, f64(gb), f64(wb), with_bound=True)
        err = oracle.max_normalised_error(f64(dx), ref, bound)
    else:
        dw, _ = F.conv2d_wgrad(xb, gb, tuple(w.shape), sh.stride, sh.pad, sh.dil, "NHWC",
                               with_bias=False)
        F.device_error()
        ref, bound = oracle.conv2d_wgrad(p, f64(xb), f64(gb), with_bound=True)
        err = oracle.max_normalised_error(f64(dw), ref, bound)
    assert err <= TOL_ACC32, (op, err, best.block_n, best.algo, best.split_k)
    return prob, best


@pytest.mark.parametrize("op", [B.GBCONV_OP_FWD, B.GBCONV_OP_DGRAD, B.GBCONV_OP_WGRAD],
                         ids=["fwd", "dgrad", "wgrad"])
@pytest.mark.parametrize("si", range(len(SHAPES)))
def test_tune_stores_a_candidate_that_matches_the_oracle(op, si):
    _tune_and_run(op, SHAPES[si], seed=120 + si)


def test_tune_cache_round_trip(tmp_path):
    tuned = [_tune_and_run(op, SHAPES[0], seed=130) for op in
             (B.GBCONV_OP_FWD, B.GBCONV_OP_DGRAD, B.GBCONV_OP_WGRAD)]
    path = os.path.join(str(tmp_path), "tune.json")
    B.check(B.gbconv_tune_cache_save(path), "save")
    B.gbconv_shutdown()  # clears the table
    B.check(B.gbconv_tune_cache_load(path), "load")
    for (prob, best), op in zip(tuned, (B.GBCONV_OP_FWD, B.GBCONV_OP_DGRAD, B.GBCONV_OP_WGRAD)):
        s, c = B.gbconv_get_config(op, prob)
        B.check(s, "get_config")
        assert _same(c, best), op
