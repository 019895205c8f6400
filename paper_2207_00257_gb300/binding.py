"""ctypes binding of include/gbconv.h -- argument marshalling only.

Every function here has the C name and C argument order; pointers are Python
ints (device addresses) and the stream is a cudaStream_t as an int. The
library is loaded from this package directory; if it is missing the import of
any entry point raises, so there is no silent fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

from ._build import LIB

GBCONV_OK = 0
GBCONV_ERR_INVALID_ARG = 1
GBCONV_ERR_UNSUPPORTED = 2
GBCONV_ERR_ALIGNMENT = 3
GBCONV_ERR_WORKSPACE = 4
GBCONV_ERR_CUDA = 5
GBCONV_ERR_TIMEOUT = 6

GBCONV_F32, GBCONV_BF16, GBCONV_E4M3 = 0, 1, 2
GBCONV_NCHW, GBCONV_NHWC = 0, 1
GBCONV_OP_FWD, GBCONV_OP_DGRAD, GBCONV_OP_WGRAD, GBCONV_OP_GROUPED = 0, 1, 2, 3
GBCONV_FLAG_BIAS, GBCONV_FLAG_RELU = 1, 2
GBCONV_DEBUG_WAIT_LIMIT_NS, GBCONV_DEBUG_SKIP_LOADS = 1, 2
GBCONV_ALGO_AUTO, GBCONV_ALGO_IM2COL, GBCONV_ALGO_SHIFT, GBCONV_ALGO_SHIFT_T = 0, 1, 2, 3
GBCONV_ALGO_SIMT = 4
GBCONV_ALGO_PBAND, GBCONV_ALGO_PBAND_PAIR = 5, 6

# every symbol include/gbconv.h declares
EXPORTS = [
    "gbconv_output_dims", "gbconv_workspace_size", "conv2d_fwd", "conv2d_dgrad",
    "conv2d_wgrad", "conv2d_grouped", "gbconv_quantize_e4m3", "gbconv_get_config",
    "gbconv_set_config", "gbconv_tune", "gbconv_tune_cache_save", "gbconv_tune_cache_load",
    "gbconv_get_device_error", "gbconv_status_string", "gbconv_debug_set", "gbconv_version",
    "gbconv_shutdown", "conv2d_dgrad_noalloc", "conv2d_fwd_fused", "gbconv_bn_fold",
    "gbconv_nll_workspace_size", "gbconv_nll_loss_fwd", "gbconv_nll_loss_bwd",
    "gbconv_relu_grad", "gbconv_measure_ffma_tflops",
]


class gbconv_problem_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("N", "C", "H", "W", "K", "R", "S", "stride_h", "stride_w", "pad_h", "pad_w",
                 "dil_h", "dil_w", "in_dtype", "out_dtype", "layout")] + [("flags", ctypes.c_uint32),
                                                                          ("groups", ctypes.c_int32)]


class gbconv_config_t(ctypes.Structure):
    _fields_ = [("block_n", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("split_k", ctypes.c_int32), ("raster", ctypes.c_int32),
                ("algo", ctypes.c_int32)]


class GbconvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_PROB = ctypes.POINTER(gbconv_problem_t)
_CFG = ctypes.POINTER(gbconv_config_t)

_SIGS = {
    "gbconv_output_dims": (ctypes.c_int, [_PROB, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "gbconv_workspace_size": (ctypes.c_int, [ctypes.c_int32, _PROB,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "conv2d_fwd": (ctypes.c_int, [_PROB, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "conv2d_dgrad": (ctypes.c_int, [_PROB, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "conv2d_wgrad": (ctypes.c_int, [_PROB, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "conv2d_grouped": (ctypes.c_int, [ctypes.c_int32, _PROB, _PP, _PP, _PP, _PP, _P,
                                      ctypes.c_size_t, _P]),
    "gbconv_quantize_e4m3": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                            _P, _P, _P]),
    "gbconv_get_config": (ctypes.c_int, [ctypes.c_int32, _PROB, _CFG]),
    "gbconv_set_config": (ctypes.c_int, [ctypes.c_int32, _PROB, _CFG]),
    "gbconv_tune": (ctypes.c_int, [ctypes.c_int32, _PROB, _P, _P, _P, _P, _P, ctypes.c_size_t,
                                   ctypes.c_int32, _P, _CFG]),
    "gbconv_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "gbconv_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "gbconv_get_device_error": (ctypes.c_int, [_P]),
    "gbconv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gbconv_debug_set": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "gbconv_version": (ctypes.c_int32, []),
    "gbconv_shutdown": (None, []),
    "conv2d_dgrad_noalloc": (ctypes.c_int, [_PROB, _P, _P, _P, _P]),
    "conv2d_fwd_fused": (ctypes.c_int, [_PROB, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        ctypes.c_size_t, _P]),
    "gbconv_bn_fold": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_float, _P, _P, _P,
                                      _P]),
    "gbconv_relu_grad": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32,
                                        ctypes.c_int64, _P]),
    "gbconv_measure_ffma_tflops": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                                  _P]),
    "gbconv_nll_workspace_size": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "gbconv_nll_loss_fwd": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int32, _P, _P, _P,
                                           ctypes.c_size_t, _P]),
    "gbconv_nll_loss_bwd": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int32, _P, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """The loaded libgbconv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(
                    f"libgbconv.so not found at {LIB}: build it first "
                    "(python -m paper_2207_00257_gb300._build)")
            L = ctypes.CDLL(LIB)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def lib_path() -> str:
    return LIB


def status_string(status: int) -> str:
    return lib().gbconv_status_string(int(status)).decode()


def check(status: int, where: str):
    if status != GBCONV_OK:
        raise GbconvError(status, where)


def _vp(v):
    return None if v is None or v == 0 else ctypes.c_void_p(int(v))


def problem(N, C, H, W, K, R, S, stride=(1, 1), pad=(0, 0), dil=(1, 1), in_dtype=GBCONV_BF16,
            out_dtype=GBCONV_BF16, layout=GBCONV_NHWC, flags=0, groups=1) -> gbconv_problem_t:
    st = (stride, stride) if isinstance(stride, int) else tuple(stride)
    pd = (pad, pad) if isinstance(pad, int) else tuple(pad)
    dl = (dil, dil) if isinstance(dil, int) else tuple(dil)
    return gbconv_problem_t(N, C, H, W, K, R, S, st[0], st[1], pd[0], pd[1], dl[0], dl[1],
                            in_dtype, out_dtype, layout, flags, groups)


# ---- the entry points, C names, C argument order ----

def gbconv_output_dims(prob):
    P, Q = ctypes.c_int32(), ctypes.c_int32()
    s = lib().gbconv_output_dims(ctypes.byref(prob), ctypes.byref(P), ctypes.byref(Q))
    return s, P.value, Q.value


def gbconv_workspace_size(op, prob):
    b = ctypes.c_size_t()
    s = lib().gbconv_workspace_size(op, ctypes.byref(prob), ctypes.byref(b))
    return s, b.value


def conv2d_fwd(prob, x, w, bias, x_scale, w_scale, y, ws, ws_bytes, stream):
    return lib().conv2d_fwd(ctypes.byref(prob), _vp(x), _vp(w), _vp(bias), _vp(x_scale),
                            _vp(w_scale), _vp(y), _vp(ws), ws_bytes, _vp(stream))


def conv2d_fwd_fused(prob, x, w, bias, scale, residual, x_scale, w_scale, y, ws, ws_bytes,
                     stream):
    return lib().conv2d_fwd_fused(ctypes.byref(prob), _vp(x), _vp(w), _vp(bias), _vp(scale),
                                  _vp(residual), _vp(x_scale), _vp(w_scale), _vp(y), _vp(ws),
                                  ws_bytes, _vp(stream))


def gbconv_bn_fold(K, gamma, bn_beta, mean, var, eps, bias, scale, shift, stream):
    return lib().gbconv_bn_fold(int(K), _vp(gamma), _vp(bn_beta), _vp(mean), _vp(var),
                                float(eps), _vp(bias), _vp(scale), _vp(shift), _vp(stream))


def gbconv_nll_workspace_size(N):
    n = ctypes.c_size_t(0)
    s = lib().gbconv_nll_workspace_size(int(N), ctypes.byref(n))
    return s, n.value


def gbconv_nll_loss_fwd(logp, target, weight, N, C, ignore_index, reduction, out, total_weight,
                        ws, ws_bytes, stream):
    return lib().gbconv_nll_loss_fwd(_vp(logp), _vp(target), _vp(weight), int(N), int(C),
                                     int(ignore_index), int(reduction), _vp(out),
                                     _vp(total_weight), _vp(ws), ws_bytes, _vp(stream))


def gbconv_nll_loss_bwd(grad_out, target, weight, N, C, ignore_index, reduction, total_weight,
                        grad_in, stream):
    return lib().gbconv_nll_loss_bwd(_vp(grad_out), _vp(target), _vp(weight), int(N), int(C),
                                     int(ignore_index), int(reduction), _vp(total_weight),
                                     _vp(grad_in), _vp(stream))


def conv2d_dgrad(prob, dy, w, dx, ws, ws_bytes, stream):
    return lib().conv2d_dgrad(ctypes.byref(prob), _vp(dy), _vp(w), _vp(dx), _vp(ws), ws_bytes,
                              _vp(stream))


def conv2d_wgrad(prob, x, dy, dw, db, ws, ws_bytes, stream):
    return lib().conv2d_wgrad(ctypes.byref(prob), _vp(x), _vp(dy), _vp(dw), _vp(db), _vp(ws),
                              ws_bytes, _vp(stream))


def conv2d_grouped(count, probs, x, w, bias, y, ws, ws_bytes, stream):
    """probs: sequence of gbconv_problem_t; x, w, bias, y: sequences of device addresses."""
    n = max(int(count), 0)
    arr = (gbconv_problem_t * n)(*probs[:n])

    def ptrs(seq):
        return (ctypes.c_void_p * n)(*[int(v) if v else None for v in seq[:n]])

    return lib().conv2d_grouped(count, arr, ptrs(x), ptrs(w), ptrs(bias) if bias else None,
                                ptrs(y), _vp(ws), ws_bytes, _vp(stream))


def gbconv_quantize_e4m3(inp, in_dtype, rows, length, out, scale, stream):
    return lib().gbconv_quantize_e4m3(_vp(inp), in_dtype, rows, length, _vp(out), _vp(scale),
                                      _vp(stream))


def gbconv_relu_grad(y, y_dtype, g, g_dtype, g_out, out_dtype, n, stream):
    return lib().gbconv_relu_grad(_vp(y), y_dtype, _vp(g), g_dtype, _vp(g_out), out_dtype, n,
                                  _vp(stream))


def gbconv_get_config(op, prob):
    c = gbconv_config_t()
    s = lib().gbconv_get_config(op, ctypes.byref(prob), ctypes.byref(c))
    return s, c


def gbconv_set_config(op, prob, cfg):
    return lib().gbconv_set_config(op, ctypes.byref(prob), ctypes.byref(cfg))


def gbconv_tune(op, prob, a, b, bias, out, ws, ws_bytes, reps, stream):
    c = gbconv_config_t()
    s = lib().gbconv_tune(op, ctypes.byref(prob), _vp(a), _vp(b), _vp(bias), _vp(out), _vp(ws),
                          ws_bytes, reps, _vp(stream), ctypes.byref(c))
    return s, c


def gbconv_tune_cache_save(path: str):
    return lib().gbconv_tune_cache_save(path.encode())


def gbconv_tune_cache_load(path: str):
    return lib().gbconv_tune_cache_load(path.encode())


def gbconv_get_device_error(stream):
    return lib().gbconv_get_device_error(_vp(stream))


def gbconv_status_string(status):
    return status_string(status)


def gbconv_debug_set(key, value):
    return lib().gbconv_debug_set(key, value)


def gbconv_measure_ffma_tflops(iters, stream):
    v = ctypes.c_double(0.0)
    s = lib().gbconv_measure_ffma_tflops(iters, ctypes.byref(v), _vp(stream))
    return s, v.value


def gbconv_version():
    return lib().gbconv_version()


def gbconv_shutdown():
    lib().gbconv_shutdown()


GBCONV_DGRAD_STATIC_SCRATCH_BYTES = 8 * 1024 * 1024


def conv2d_dgrad_noalloc(prob, dy, w, dx, stream):
    return lib().conv2d_dgrad_noalloc(ctypes.byref(prob), _vp(dy), _vp(w), _vp(dx), _vp(stream))
