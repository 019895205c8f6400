"""GPU parity of the negative log-likelihood loss (forward and gradient)
against the FP64 oracle on the same fp32 log-probabilities."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00257_gb300 import binding as B
from paper_2207_00257_gb300 import functional as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _inputs(N, C, seed, weighted, n_ignored=3):
    g = torch.Generator().manual_seed(seed)
    logp = torch.log_softmax(torch.randn(N, C, generator=g), dim=1)
    t = torch.randint(0, C, (N,), generator=g)
    if N > n_ignored:
        t[torch.randperm(N, generator=g)[:n_ignored]] = -100
    w = (torch.rand(C, generator=g) + 0.5) if weighted else None
    return logp, t, w


# FP32 tree reduction of up to 2^17 terms: log2(N) * 2^-24 of the absolute sum
TOL = 2e-6


@pytest.mark.parametrize("N,C", [(37, 11), (5000, 10), (100000, 1000), (1, 3)])
@pytest.mark.parametrize("reduction", ["none", "mean", "sum"])
@pytest.mark.parametrize("weighted", [False, True])
def test_nll_forward_and_gradient(N, C, reduction, weighted):
    logp, t, w = _inputs(N, C, 100 + N, weighted)
    dev = "cuda"
    out, tw = F.nll_loss(logp.to(dev), t.to(dev), w.to(dev) if weighted else None, -100, reduction)
    F.device_error()
    ref, tw_ref = oracle.nll_loss(logp.double(), t, w.double() if weighted else None, -100,
                                  reduction)
    lp = logp.double().numpy()
    tn = t.numpy()
    wn = w.double().numpy() if weighted else np.ones(C)
    counted = tn != -100
    terms = np.zeros(N)
    terms[counted] = np.abs(wn[tn[counted]] * lp[np.nonzero(counted)[0], tn[counted]])
    if reduction == "none":
        assert np.max(np.abs(out.double().cpu().numpy() - ref) / np.maximum(terms, 1e-30)) < 1e-6
    else:
        scale = terms.sum() / (tw_ref if reduction == "mean" else 1.0)
        assert abs(float(out) - ref[0]) <= TOL * max(scale, 1e-30)
    assert abs(float(tw) - tw_ref) <= TOL * max(tw_ref, 1e-30)
    g = torch.Generator().manual_seed(7)
    go = torch.randn(N if reduction == "none" else 1, generator=g)
    gi = F.nll_loss_backward(go.to(dev), t.to(dev), tw, C, w.to(dev) if weighted else None, -100,
                             reduction)
    F.device_error()
    gref = oracle.nll_loss_grad(go.double(), t, N, C, w.double() if weighted else None, -100,
                                reduction, tw_ref)
    assert np.max(np.abs(gi.double().cpu().numpy() - gref)) <= 1e-6 * max(np.abs(gref).max(), 1e-30)
    assert np.count_nonzero(gi.cpu().numpy()) <= int(counted.sum())


def test_nll_deterministic():
    logp, t, w = _inputs(70000, 100, 5, True)
    dev = "cuda"
    a, _ = F.nll_loss(logp.to(dev), t.to(dev), w.to(dev))
    b, _ = F.nll_loss(logp.to(dev), t.to(dev), w.to(dev))
    assert torch.equal(a, b)


def test_nll_all_ignored_mean_is_nan():
    logp, t, _ = _inputs(10, 4, 6, False)
    t[:] = -100
    out, tw = F.nll_loss(logp.cuda(), t.cuda())
    F.device_error()
    assert float(tw) == 0.0 and np.isnan(float(out))


def test_nll_bad_target_reports_and_is_ignored():
    logp, t, _ = _inputs(50, 5, 8, False, n_ignored=0)
    t[7] = 9  # outside [0, 5)
    out, tw = F.nll_loss(logp.cuda(), t.cuda(), reduction="sum")
    assert B.gbconv_get_device_error(torch.cuda.current_stream().cuda_stream) == \
        B.GBCONV_ERR_INVALID_ARG
    t2 = t.clone()
    t2[7] = -100
    ref, _ = oracle.nll_loss(logp.double(), t2, reduction="sum")
    assert abs(float(out) - ref[0]) <= 1e-5 * abs(ref[0])
    assert B.gbconv_get_device_error(torch.cuda.current_stream().cuda_stream) == B.GBCONV_OK


def test_nll_argument_checks():
    st = torch.cuda.current_stream().cuda_stream
    assert B.gbconv_nll_loss_fwd(0, 0, 0, -1, 3, -100, 1, 16, 32, 64, 64, st) == \
        B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_nll_loss_fwd(16, 32, 0, 10, 3, -100, 3, 16, 32, 64, 64, st) == \
        B.GBCONV_ERR_INVALID_ARG
    s, n = B.gbconv_nll_workspace_size(10)
    assert s == B.GBCONV_OK and n > 0
    assert B.gbconv_nll_loss_fwd(16, 32, 0, 10, 3, -100, 1, 48, 64, 0, 0, st) == \
        B.GBCONV_ERR_WORKSPACE
