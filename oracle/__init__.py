"""FP64 CPU oracle for dense 2D convolution -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package. The product library
(``paper_2207_00257_gb300``) never imports it, and it never imports the
product library: the two share no code. Inputs reach both sides from
``paper_2207_00257_gb300.synth`` (seeded generators only, no convolution
arithmetic).

The arithmetic lives in ``oracle.c`` (plain C, double precision, six nested
loops: the definition of the convolution as the paper's Sec. 1 / Sec. 5.A
describe PyTorch's native CPU kernel, and its forward and backward passes as
Sec. 5.B lists them). This module only compiles it with gcc and marshals numpy
arrays through ctypes.

Layouts: ``"NCHW"`` (filters KCRS) or ``"NHWC"`` (filters KRSC).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no vendor code involved)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_output_dims.argtypes = [_i64p, _i64p, _i64p]
            lib.oracle_conv2d_fwd.argtypes = [_i64p, _f64p, _f64p, _f64p, ctypes.c_int,
                                              _i64p, ctypes.c_int64, _f64p, _f64p, ctypes.c_int]
            lib.oracle_conv2d_dgrad.argtypes = [_i64p, _f64p, _f64p, _i64p, ctypes.c_int64,
                                                _f64p, _f64p, ctypes.c_int]
            lib.oracle_conv2d_wgrad.argtypes = [_i64p, _f64p, _f64p, _i64p, ctypes.c_int64,
                                                _f64p, _f64p, ctypes.c_int]
            lib.oracle_conv2d_bgrad.argtypes = [_i64p, _f64p, _f64p, _f64p]
            lib.oracle_conv2d_fwd_fused.argtypes = [_i64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                                    ctypes.c_int, _i64p, ctypes.c_int64, _f64p,
                                                    _f64p, ctypes.c_int]
            lib.oracle_bn_fold.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p,
                                           ctypes.c_double, _f64p, _f64p, _f64p]
            lib.oracle_bn_fold.restype = None
            lib.oracle_nll_loss_fwd.argtypes = [_f64p, _i64p, _f64p, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                _f64p, _f64p]
            lib.oracle_nll_loss_bwd.argtypes = [_f64p, _i64p, _f64p, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_double, _f64p]
            lib.oracle_nll_loss_fwd.restype = ctypes.c_int
            lib.oracle_nll_loss_bwd.restype = ctypes.c_int
            lib.oracle_round_bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            lib.oracle_bf16_to_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            lib.oracle_quant_e4m3.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            lib.oracle_e4m3_to_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            lib.oracle_scale_quant_e4m3.argtypes = [ctypes.c_void_p, ctypes.c_int64,
                                                    ctypes.c_int64, ctypes.c_void_p,
                                                    ctypes.c_void_p]
            for f in ("oracle_output_dims", "oracle_conv2d_fwd", "oracle_conv2d_dgrad",
                      "oracle_conv2d_wgrad", "oracle_conv2d_bgrad", "oracle_conv2d_fwd_fused"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


class Conv:
    """Problem description: per-axis stride (u, v), padding and dilation."""

    def __init__(self, N, C, H, W, K, R, S, stride=1, pad=0, dil=1, layout="NCHW", groups=1):
        su, sv = (stride, stride) if np.isscalar(stride) else stride
        ph, pw = (pad, pad) if np.isscalar(pad) else pad
        dh, dw = (dil, dil) if np.isscalar(dil) else dil
        if layout not in ("NCHW", "NHWC"):
            raise ValueError(layout)
        self.N, self.C, self.H, self.W, self.K, self.R, self.S = N, C, H, W, K, R, S
        self.u, self.v, self.ph, self.pw, self.dh, self.dw = su, sv, ph, pw, dh, dw
        self.layout = layout
        self.G = groups
        self.d = np.array([N, C, H, W, K, R, S, su, sv, ph, pw, dh, dw,
                           0 if layout == "NCHW" else 1, groups], dtype=np.int64)
        P, Q = ctypes.c_int64(), ctypes.c_int64()
        if _load().oracle_output_dims(_ptr(self.d, _i64p), ctypes.byref(P), ctypes.byref(Q)):
            raise ValueError("invalid convolution dimensions")
        self.P, self.Q = P.value, Q.value

    # shapes in the problem's layout
    @property
    def x_shape(self):
        return ((self.N, self.C, self.H, self.W) if self.layout == "NCHW"
                else (self.N, self.H, self.W, self.C))

    @property
    def w_shape(self):  # C/G channels per output channel
        cg = self.C // self.G
        return ((self.K, cg, self.R, self.S) if self.layout == "NCHW"
                else (self.K, self.R, self.S, cg))

    @property
    def y_shape(self):
        return ((self.N, self.K, self.P, self.Q) if self.layout == "NCHW"
                else (self.N, self.P, self.Q, self.K))

    @property
    def flops(self):
        return 2 * self.N * self.K * self.P * self.Q * (self.C // self.G) * self.R * self.S


def _ptr(a, typ):
    return a.ctypes.data_as(typ)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _idx(idx):
    if idx is None:
        return None, 0
    i = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    return i, i.size


def conv2d_fwd(p: Conv, x, w, b=None, relu=False, idx=None, nthreads=0, with_bound=False):
    """y (or y at the linear output indices ``idx``) in float64."""
    lib = _load()
    x, w = _f64(x), _f64(w)
    assert x.size == int(np.prod(p.x_shape)) and w.size == int(np.prod(p.w_shape))
    bb = _f64(b) if b is not None else None
    i, n = _idx(idx)
    out = np.empty(n if i is not None else p.y_shape, dtype=np.float64)
    bound = np.empty_like(out) if with_bound else None
    rc = lib.oracle_conv2d_fwd(_ptr(p.d, _i64p), _ptr(x, _f64p), _ptr(w, _f64p),
                               _ptr(bb, _f64p) if bb is not None else None, int(bool(relu)),
                               _ptr(i, _i64p) if i is not None else None, n,
                               _ptr(out, _f64p), _ptr(bound, _f64p) if with_bound else None,
                               int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_conv2d_fwd failed ({rc})")
    return (out, bound) if with_bound else out


def conv2d_fwd_fused(p: Conv, x, w, alpha=None, beta=None, z=None, relu=False, idx=None,
                     nthreads=0, with_bound=False):
    """y = act(alpha[k] * conv + beta[k] + z) in float64 (the layers after a
    ResNet-50 convolution, Sec. 5.B: batch normalisation folded into
    (alpha, beta), the tensor add of the residual z). alpha, beta, z may be
    None; z has y's shape and layout."""
    lib = _load()
    x, w = _f64(x), _f64(w)
    assert x.size == int(np.prod(p.x_shape)) and w.size == int(np.prod(p.w_shape))
    al = _f64(alpha) if alpha is not None else None
    be = _f64(beta) if beta is not None else None
    zz = _f64(z) if z is not None else None
    if zz is not None:
        assert zz.size == int(np.prod(p.y_shape))
    i, n = _idx(idx)
    out = np.empty(n if i is not None else p.y_shape, dtype=np.float64)
    bound = np.empty_like(out) if with_bound else None
    opt = lambda a: _ptr(a, _f64p) if a is not None else None
    rc = lib.oracle_conv2d_fwd_fused(_ptr(p.d, _i64p), _ptr(x, _f64p), _ptr(w, _f64p), opt(al),
                                     opt(be), opt(zz), int(bool(relu)),
                                     _ptr(i, _i64p) if i is not None else None, n,
                                     _ptr(out, _f64p), _ptr(bound, _f64p) if with_bound else None,
                                     int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_conv2d_fwd_fused failed ({rc})")
    return (out, bound) if with_bound else out


def bn_fold(gamma, bn_beta, mean, var, eps, bias=None):
    """Inference batch normalisation after a convolution with bias b, folded
    into the fused forward's per-channel (alpha, beta), in float64."""
    g, bb, m, v = (_f64(a) for a in (gamma, bn_beta, mean, var))
    K = g.size
    b = _f64(bias) if bias is not None else None
    alpha, beta = np.empty(K), np.empty(K)
    _load().oracle_bn_fold(K, _ptr(g, _f64p), _ptr(bb, _f64p), _ptr(m, _f64p), _ptr(v, _f64p),
                           float(eps), _ptr(b, _f64p) if b is not None else None,
                           _ptr(alpha, _f64p), _ptr(beta, _f64p))
    return alpha, beta


def conv2d_dgrad(p: Conv, g, w, idx=None, nthreads=0, with_bound=False):
    """dL/dx for L = sum(g * y), in float64 (full x shape, or at ``idx``)."""
    lib = _load()
    g, w = _f64(g), _f64(w)
    i, n = _idx(idx)
    out = np.empty(n if i is not None else p.x_shape, dtype=np.float64)
    bound = np.empty_like(out) if with_bound else None
    rc = lib.oracle_conv2d_dgrad(_ptr(p.d, _i64p), _ptr(g, _f64p), _ptr(w, _f64p),
                                 _ptr(i, _i64p) if i is not None else None, n,
                                 _ptr(out, _f64p), _ptr(bound, _f64p) if with_bound else None,
                                 int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_conv2d_dgrad failed ({rc})")
    return (out, bound) if with_bound else out


def conv2d_wgrad(p: Conv, x, g, idx=None, nthreads=0, with_bound=False):
    """dL/dw for L = sum(g * y), in float64 (full w shape, or at ``idx``)."""
    lib = _load()
    x, g = _f64(x), _f64(g)
    i, n = _idx(idx)
    out = np.empty(n if i is not None else p.w_shape, dtype=np.float64)
    bound = np.empty_like(out) if with_bound else None
    rc = lib.oracle_conv2d_wgrad(_ptr(p.d, _i64p), _ptr(x, _f64p), _ptr(g, _f64p),
                                 _ptr(i, _i64p) if i is not None else None, n,
                                 _ptr(out, _f64p), _ptr(bound, _f64p) if with_bound else None,
                                 int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_conv2d_wgrad failed ({rc})")
    return (out, bound) if with_bound else out


def conv2d_bgrad(p: Conv, g, with_bound=False):
    """dL/db[k] = sum over n, p, q of g."""
    lib = _load()
    g = _f64(g)
    out = np.empty(p.K, dtype=np.float64)
    bound = np.empty_like(out)
    rc = lib.oracle_conv2d_bgrad(_ptr(p.d, _i64p), _ptr(g, _f64p), _ptr(out, _f64p),
                                 _ptr(bound, _f64p))
    if rc:
        raise RuntimeError(f"oracle_conv2d_bgrad failed ({rc})")
    return (out, bound) if with_bound else out


# ---- quantisers (binary32 in; codes and exact float64 values out) ----

def round_bf16_bits(a) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest even."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    out = np.empty(a.shape, dtype=np.uint16)
    _load().oracle_round_bf16(a.ctypes.data, out.ctypes.data, a.size)
    return out


def bf16_bits_to_f64(bits) -> np.ndarray:
    bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint16))
    out = np.empty(bits.shape, dtype=np.float64)
    _load().oracle_bf16_to_f64(bits.ctypes.data, out.ctypes.data, bits.size)
    return out


def round_bf16(a) -> np.ndarray:
    """FP32 values rounded to BF16, returned exactly as float64."""
    return bf16_bits_to_f64(round_bf16_bits(a))


def quant_e4m3(a) -> np.ndarray:
    """FP32 -> E4M3 codes (uint8), round to nearest even, saturating to +-448."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    out = np.empty(a.shape, dtype=np.uint8)
    _load().oracle_quant_e4m3(a.ctypes.data, out.ctypes.data, a.size)
    return out


def e4m3_to_f64(codes) -> np.ndarray:
    codes = np.ascontiguousarray(np.asarray(codes, dtype=np.uint8))
    out = np.empty(codes.shape, dtype=np.float64)
    _load().oracle_e4m3_to_f64(codes.ctypes.data, out.ctypes.data, codes.size)
    return out


def scale_quant_e4m3(a, rows: int):
    """Per-row FP8 preparation: s = max|row|/448 (floored at 1e-12), q = E4M3(row/s).

    ``a`` is viewed as ``rows`` contiguous groups. Returns (codes, scales)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    assert a.size % rows == 0
    out = np.empty(a.shape, dtype=np.uint8)
    scales = np.empty(rows, dtype=np.float32)
    _load().oracle_scale_quant_e4m3(a.ctypes.data, rows, a.size // rows, out.ctypes.data,
                                    scales.ctypes.data)
    return out, scales


def max_normalised_error(got, ref, bound) -> float:
    """max |got - ref| / max(bound, 1e-30): the error the tolerances are quoted in."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bound = np.maximum(np.asarray(bound, dtype=np.float64), 1e-30)
    if got.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref) / bound))


# ---- the rectifier after a convolution (Sec. 5.B, backward pass) ----

def relu_grad(y, g) -> np.ndarray:
    """Gradient through y = max(z, 0) in float64: g where y > 0, else 0
    (the derivative of the rectifier is 1 for z > 0 and 0 for z < 0; at
    z = 0 the zero branch, as PyTorch's threshold backward takes it)."""
    y = np.asarray(y, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    return np.where(y > 0, g, 0.0)


# ---- negative log-likelihood loss (Sec. 5.B) ----

NLL_REDUCTIONS = {"none": 0, "mean": 1, "sum": 2}


def nll_loss(logp, target, weight=None, ignore_index=-100, reduction="mean"):
    """The ClassNLLCriterion forward in float64: returns (out, total_weight);
    out has N values for reduction 'none', else one."""
    lp = _f64(logp)
    N, C = lp.shape
    t = np.ascontiguousarray(np.asarray(target, dtype=np.int64))
    wt = _f64(weight) if weight is not None else None
    red = NLL_REDUCTIONS[reduction]
    out = np.empty(N if red == 0 else 1)
    tw = np.empty(1)
    rc = _load().oracle_nll_loss_fwd(_ptr(lp, _f64p), _ptr(t, _i64p),
                                     _ptr(wt, _f64p) if wt is not None else None, N, C,
                                     int(ignore_index), red, _ptr(out, _f64p), _ptr(tw, _f64p))
    if rc:
        raise ValueError("target outside [0, C) and not ignore_index")
    return out, float(tw[0])


def nll_loss_grad(grad_out, target, N, C, weight=None, ignore_index=-100, reduction="mean",
                  total_weight=1.0):
    """The ClassNLLCriterion gradient with respect to logp, [N][C] float64."""
    g = _f64(np.atleast_1d(grad_out))
    t = np.ascontiguousarray(np.asarray(target, dtype=np.int64))
    wt = _f64(weight) if weight is not None else None
    out = np.empty((N, C))
    rc = _load().oracle_nll_loss_bwd(_ptr(g, _f64p), _ptr(t, _i64p),
                                     _ptr(wt, _f64p) if wt is not None else None, N, C,
                                     int(ignore_index), NLL_REDUCTIONS[reduction],
                                     float(total_weight), _ptr(out, _f64p))
    if rc:
        raise ValueError("target outside [0, C) and not ignore_index")
    return out
