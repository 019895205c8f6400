"""Torch-facing helpers over the C ABI: shape bookkeeping, output allocation
through torch (PyTorch supplies device memory and streams only), status checks,
and the autograd Function. Every arithmetic step runs in libgbconv's kernels.
"""
from __future__ import annotations

import torch

from . import binding as B

_DT = {torch.float32: B.GBCONV_F32, torch.bfloat16: B.GBCONV_BF16,
       torch.float8_e4m3fn: B.GBCONV_E4M3, torch.uint8: B.GBCONV_E4M3}
_TORCH = {B.GBCONV_F32: torch.float32, B.GBCONV_BF16: torch.bfloat16}


def _pair(v):
    return (v, v) if isinstance(v, int) else tuple(v)


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _check_dev(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("gbconv expects contiguous CUDA tensors")


def make_problem(x, w, stride=1, padding=0, dilation=1, layout="NHWC", out_dtype=None,
                 bias=False, relu=False, groups=1):
    lay = B.GBCONV_NHWC if layout == "NHWC" else B.GBCONV_NCHW
    if layout == "NHWC":
        N, H, W, C = x.shape
        K, R, S, C2 = w.shape
    else:
        N, C, H, W = x.shape
        K, C2, R, S = w.shape
    if C != C2 * groups:
        raise ValueError(f"channel mismatch: x has {C}, w has {C2} per group x {groups} groups")
    ind = _DT[x.dtype]
    outd = _DT[out_dtype] if out_dtype is not None else (B.GBCONV_BF16 if ind == B.GBCONV_E4M3 else ind)
    flags = (B.GBCONV_FLAG_BIAS if bias else 0) | (B.GBCONV_FLAG_RELU if relu else 0)
    return B.problem(N, C, H, W, K, R, S, _pair(stride), _pair(padding), _pair(dilation), ind,
                     outd, lay, flags, groups)


def out_shape(prob, layout):
    s, P, Q = B.gbconv_output_dims(prob)
    B.check(s, "gbconv_output_dims")
    return (prob.N, P, Q, prob.K) if layout == "NHWC" else (prob.N, prob.K, P, Q)


def conv2d(x, w, bias=None, stride=1, padding=0, dilation=1, relu=False, layout="NHWC",
           out_dtype=None, x_scale=None, w_scale=None, out=None, groups=1):
    """Forward convolution through conv2d_fwd. For E4M3 inputs pass the fp32
    scales (x_scale: 1 element, w_scale: K elements) from quantize_e4m3.
    groups > 1: channel groups (w holds C/groups channels per output channel)."""
    _check_dev(x, w, bias, x_scale, w_scale)
    prob = make_problem(x, w, stride, padding, dilation, layout, out_dtype, bias is not None, relu,
                        groups)
    if out is None:
        out = torch.empty(out_shape(prob, layout), dtype=_TORCH[prob.out_dtype], device=x.device)
    ws, nbytes = workspace(B.GBCONV_OP_FWD, prob, x.device)
    s = B.conv2d_fwd(prob, x.data_ptr(), w.data_ptr(), bias.data_ptr() if bias is not None else 0,
                     x_scale.data_ptr() if x_scale is not None else 0,
                     w_scale.data_ptr() if w_scale is not None else 0, out.data_ptr(),
                     ws.data_ptr() if nbytes else 0, nbytes, _stream())
    B.check(s, "conv2d_fwd")
    return out


def conv2d_fused(x, w, bias=None, scale=None, residual=None, stride=1, padding=0, dilation=1,
                 relu=False, layout="NHWC", out_dtype=None, x_scale=None, w_scale=None, out=None,
                 groups=1):
    """y = act(scale[k] * conv(x, w) + bias[k] + residual) through
    conv2d_fwd_fused (batch normalisation folded into scale/bias with
    bn_fold; residual of y's shape and dtype, may be ``out`` itself)."""
    _check_dev(x, w, bias, scale, residual, x_scale, w_scale)
    prob = make_problem(x, w, stride, padding, dilation, layout, out_dtype, bias is not None, relu,
                        groups)
    if out is None:
        out = torch.empty(out_shape(prob, layout), dtype=_TORCH[prob.out_dtype], device=x.device)
    ptr = lambda t: t.data_ptr() if t is not None else 0
    ws, nbytes = workspace(B.GBCONV_OP_FWD, prob, x.device)
    s = B.conv2d_fwd_fused(prob, x.data_ptr(), w.data_ptr(), ptr(bias), ptr(scale), ptr(residual),
                           ptr(x_scale), ptr(w_scale), out.data_ptr(),
                           ws.data_ptr() if nbytes else 0, nbytes, _stream())
    B.check(s, "conv2d_fwd_fused")
    return out


def bn_fold(gamma, bn_beta, mean, var, eps, bias=None):
    """Folds inference batch normalisation (after a convolution with ``bias``)
    into the fused forward's per-channel (scale, shift), on the device."""
    _check_dev(gamma, bn_beta, mean, var, bias)
    K = gamma.numel()
    scale = torch.empty(K, dtype=torch.float32, device=gamma.device)
    shift = torch.empty(K, dtype=torch.float32, device=gamma.device)
    s = B.gbconv_bn_fold(K, gamma.data_ptr(), bn_beta.data_ptr(), mean.data_ptr(), var.data_ptr(),
                         eps, bias.data_ptr() if bias is not None else 0, scale.data_ptr(),
                         shift.data_ptr(), _stream())
    B.check(s, "gbconv_bn_fold")
    return scale, shift


_NLL_RED = {"none": 0, "mean": 1, "sum": 2}


def nll_loss(logp, target, weight=None, ignore_index=-100, reduction="mean"):
    """Negative log-likelihood loss forward through gbconv_nll_loss_fwd.
    Returns (out, total_weight) as device tensors."""
    _check_dev(logp, target, weight)
    N, C = logp.shape
    red = _NLL_RED[reduction]
    out = torch.empty(N if red == 0 else 1, dtype=torch.float32, device=logp.device)
    tw = torch.empty(1, dtype=torch.float32, device=logp.device)
    s, nbytes = B.gbconv_nll_workspace_size(N)
    B.check(s, "gbconv_nll_workspace_size")
    ws = torch.empty(max(nbytes, 4), dtype=torch.uint8, device=logp.device)
    s = B.gbconv_nll_loss_fwd(logp.data_ptr(), target.data_ptr(),
                              weight.data_ptr() if weight is not None else 0, N, C, ignore_index,
                              red, out.data_ptr(), tw.data_ptr(), ws.data_ptr(), nbytes, _stream())
    B.check(s, "gbconv_nll_loss_fwd")
    return (out if red == 0 else out[0]), tw


def nll_loss_backward(grad_out, target, total_weight, C, weight=None, ignore_index=-100,
                      reduction="mean"):
    """Gradient of the loss with respect to logp through gbconv_nll_loss_bwd."""
    _check_dev(grad_out, target, total_weight, weight)
    N = target.numel()
    gi = torch.empty(N, C, dtype=torch.float32, device=target.device)
    s = B.gbconv_nll_loss_bwd(grad_out.data_ptr(), target.data_ptr(),
                              weight.data_ptr() if weight is not None else 0, N, C, ignore_index,
                              _NLL_RED[reduction], total_weight.data_ptr(), gi.data_ptr(),
                              _stream())
    B.check(s, "gbconv_nll_loss_bwd")
    return gi


def workspace(op, prob, device):
    s, nbytes = B.gbconv_workspace_size(op, prob)
    B.check(s, "gbconv_workspace_size")
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device), nbytes


def conv2d_dgrad(dy, w, x_shape, stride=1, padding=0, dilation=1, layout="NHWC", out_dtype=None,
                 groups=1):
    """dL/dx for upstream gradient dy."""
    _check_dev(dy, w)
    fake_x = torch.empty(x_shape, dtype=dy.dtype, device="meta")
    prob = make_problem(fake_x, w, stride, padding, dilation, layout, out_dtype, groups=groups)
    dx = torch.empty(x_shape, dtype=_TORCH[prob.out_dtype], device=dy.device)
    ws, nbytes = workspace(B.GBCONV_OP_DGRAD, prob, dy.device)
    s = B.conv2d_dgrad(prob, dy.data_ptr(), w.data_ptr(), dx.data_ptr(), ws.data_ptr(), nbytes,
                       _stream())
    B.check(s, "conv2d_dgrad")
    return dx


def conv2d_wgrad(x, dy, w_shape, stride=1, padding=0, dilation=1, layout="NHWC", with_bias=True,
                 groups=1):
    """(dL/dw, dL/db) in fp32 for upstream gradient dy."""
    _check_dev(x, dy)
    fake_w = torch.empty(w_shape, dtype=x.dtype, device="meta")
    prob = make_problem(x, fake_w, stride, padding, dilation, layout, groups=groups)
    dw = torch.empty(w_shape, dtype=torch.float32, device=x.device)
    db = torch.empty(prob.K, dtype=torch.float32, device=x.device) if with_bias else None
    ws, nbytes = workspace(B.GBCONV_OP_WGRAD, prob, x.device)
    s = B.conv2d_wgrad(prob, x.data_ptr(), dy.data_ptr(), dw.data_ptr(),
                       db.data_ptr() if db is not None else 0, ws.data_ptr(), nbytes, _stream())
    B.check(s, "conv2d_wgrad")
    return dw, db


def relu_grad(y, g, out_dtype=None, out=None):
    """Gradient through the ReLU of a forward with relu=True: g where y > 0,
    else 0 (gbconv_relu_grad), in ``out_dtype`` (default: g's dtype)."""
    _check_dev(y, g)
    if y.numel() != g.numel():
        raise ValueError("y and g must have the same number of elements")
    od = out_dtype if out_dtype is not None else g.dtype
    if out is None:
        out = torch.empty(g.shape, dtype=od, device=g.device)
    s = B.gbconv_relu_grad(y.data_ptr(), _DT[y.dtype], g.data_ptr(), _DT[g.dtype],
                           out.data_ptr(), _DT[out.dtype], g.numel(), _stream())
    B.check(s, "gbconv_relu_grad")
    return out


def quantize_e4m3(t, rows=1):
    """Per-group FP8 preparation: returns (codes as float8_e4m3fn, fp32 scales[rows])."""
    _check_dev(t)
    out = torch.empty(t.shape, dtype=torch.float8_e4m3fn, device=t.device)
    scale = torch.empty(rows, dtype=torch.float32, device=t.device)
    s = B.gbconv_quantize_e4m3(t.data_ptr(), _DT[t.dtype], rows, t.numel() // rows,
                               out.data_ptr(), scale.data_ptr(), _stream())
    B.check(s, "gbconv_quantize_e4m3")
    return out, scale


def conv2d_grouped(xs, ws, biases, strides, pads, relu=False, outs=None):
    """Many independent BF16 NHWC forward convolutions in one persistent launch."""
    probs, ys = [], []
    for i, (x, w) in enumerate(zip(xs, ws)):
        _check_dev(x, w)
        b = biases[i] if biases is not None else None
        p = make_problem(x, w, strides[i], pads[i], 1, "NHWC", None, b is not None, relu)
        probs.append(p)
        ys.append(outs[i] if outs is not None else
                  torch.empty(out_shape(p, "NHWC"), dtype=torch.bfloat16, device=x.device))
    bias_ptrs = [b.data_ptr() if b is not None else 0 for b in (biases or [None] * len(xs))]
    s = B.conv2d_grouped(len(probs), probs, [x.data_ptr() for x in xs], [w.data_ptr() for w in ws],
                         bias_ptrs if biases is not None else None, [y.data_ptr() for y in ys],
                         0, 0, _stream())
    B.check(s, "conv2d_grouped")
    return ys


def device_error():
    """Synchronise the current stream; raise if a bounded in-kernel wait ran out."""
    B.check(B.gbconv_get_device_error(_stream()), "device")


class Conv2dFn(torch.autograd.Function):
    """y = conv2d(x, w) + b (optionally ReLU) with hand-written backward
    kernels: conv2d_dgrad for dx and conv2d_wgrad for dw, db."""

    @staticmethod
    def forward(ctx, x, w, b, stride, padding, dilation, relu, layout, groups=1):
        y = conv2d(x, w, b, stride, padding, dilation, relu, layout, groups=groups)
        ctx.save_for_backward(x, w, y if relu else None)
        ctx.conf = (stride, padding, dilation, relu, layout, b is not None,
                    b.dtype if b is not None else None, groups)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, w, y = ctx.saved_tensors
        stride, padding, dilation, relu, layout, has_b, bdt, groups = ctx.conf
        gy = gy.contiguous()
        if relu:
            # derivative of max(., 0) (and the cast to x's dtype) in the library
            gy = relu_grad(y, gy, out_dtype=x.dtype)
        else:
            gy = gy.to(x.dtype).contiguous()
        dx = dw = db = None
        if ctx.needs_input_grad[0]:
            dx = conv2d_dgrad(gy, w, tuple(x.shape), stride, padding, dilation, layout,
                              out_dtype=x.dtype, groups=groups)
        if ctx.needs_input_grad[1] or (has_b and ctx.needs_input_grad[2]):
            dw32, db32 = conv2d_wgrad(x, gy, tuple(w.shape), stride, padding, dilation, layout,
                                      with_bias=has_b, groups=groups)
            dw = dw32.to(w.dtype)
            db = db32.to(bdt) if has_b else None
        return dx, dw, db, None, None, None, None, None, None


def conv2d_autograd(x, w, b=None, stride=1, padding=0, dilation=1, relu=False, layout="NHWC",
                    groups=1):
    return Conv2dFn.apply(x, w, b, stride, padding, dilation, relu, layout, groups)
