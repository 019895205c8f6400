// internal.h -- declarations shared by the translation units of libgbconv.
// Nothing here is part of the public ABI (include/gbconv.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbconv.h"

namespace gbc {

// A validated problem with derived sizes. Stride/pad/dilation per axis:
// (u, ph, dh) along H and (v, pw, dw) along W.
struct Dims {
    int N, C, H, W, K, R, S, P, Q;
    int u, v, ph, pw, dh, dw;
    int layout;        // GBCONV_NCHW / GBCONV_NHWC
    int in_dtype, out_dtype;
    unsigned flags;
    int G = 1;         // channel groups (C and K are the totals)
    int ldxc = 0;      // NHWC channel stride of x's pixel rows when > 0 (else C): one
    int ldyc = 0;      // group of a grouped layer run as its own problem (else K)
    long long M() const { return (long long)N * P * Q; }
    int xstride() const { return ldxc > 0 ? ldxc : C; }
    int ystride() const { return ldyc > 0 ? ldyc : K; }
};

// Parameters every kernel gets for its bounded waits and error report.
struct Guard {
    unsigned int *err;   // device error word (static __device__ variable)
    uint64_t wait_ns;    // time limit of one wait
    int skip_loads;      // test control: issue no loads (consumers then time out)
};

// Fused forward epilogue (batch normalisation folded, residual add): y =
// act(alpha[k]*conv + bias[k] + z). alpha [K] fp32 and z (y's shape, layout
// and dtype; may be y itself) are optional.
struct Fused {
    const float *alpha = nullptr;
    const void *z = nullptr;
};

// Error codes written to the device error word.
enum : unsigned { DEVERR_NONE = 0, DEVERR_TIMEOUT = 1, DEVERR_BAD_INDEX = 2 };

// api.cu
Guard make_guard();                   // current device's error word + limits
int sm_count();                       // SMs of the current device
gbconv_status_t cuda_status(cudaError_t e);

// simt.cu: CUDA-core FP32-accumulate kernels (any layout/stride/dilation).
// Forward with d.G >= 1 channel groups (one grid layer per group).
gbconv_status_t launch_simt_fwd(const Dims &d, const void *x, const void *w, const float *bias,
                                void *y, cudaStream_t st, const Fused &fz = Fused{});
// simt_fast.cu: FP32 NHWC forward with C and K multiples of 4 (16-byte vectors,
// 128 x 128 / 128 x 64 register-blocked tiles); simt_fast_supported checks
// layout, dtypes, channel counts and pointer alignment (z: residual or null).
bool simt_fast_supported(const Dims &d, const void *x, const void *w, const void *y, const void *z);
gbconv_status_t launch_simt_fast_fwd(const Dims &d, const void *x, const void *w, const float *bias,
                                     void *y, cudaStream_t st, const Fused &fz = Fused{});
// nll.cu: negative log-likelihood loss (fp32 log-probabilities [N][C]).
size_t nll_workspace_bytes(long long N);
gbconv_status_t launch_nll_fwd(const float *logp, const int64_t *target, const float *weight,
                               long long N, long long C, long long ignore_index, int reduction,
                               float *out, float *total_weight, float *ws, cudaStream_t st);
gbconv_status_t launch_nll_grad(const float *grad_out, const int64_t *target, const float *weight,
                                long long N, long long C, long long ignore_index, int reduction,
                                const float *total_weight, float *grad_in, cudaStream_t st);
// depthwise.cu: NHWC depthwise forward (G = C = K), 8 channels per thread.
bool depthwise_supported(const Dims &d);
gbconv_status_t launch_depthwise(const Dims &d, const void *x, const void *w, const float *bias,
                                 void *y, cudaStream_t st, const Fused &fz = Fused{});
gbconv_status_t launch_simt_dgrad(const Dims &d, const void *g, const void *w, void *dx,
                                  cudaStream_t st);
// Partial sums of dw per slice: ws[slice][K*C*R*S] in the filter layout.
gbconv_status_t launch_simt_wgrad_partials(const Dims &d, const void *x, const void *g,
                                           float *ws, int slices, cudaStream_t st);

// aux.cu
gbconv_status_t launch_reduce_slices(const float *ws, int slices, long long n, float *out,
                                     cudaStream_t st);
gbconv_status_t launch_bias_grad(const Dims &d, const void *g, float *db, float *ws,
                                 int slices, cudaStream_t st);
gbconv_status_t launch_rotate_filter(const Dims &d, const void *w, void *w_rot, cudaStream_t st);
// w[k][r][s][c] -> wT[c][r][s][k] (BF16)
gbconv_status_t launch_transpose_filter(const Dims &d, const void *w, void *wt, cudaStream_t st);
// out[b][j][i] = in[b][i][j], in = [B][R][Cn], 2- or 4-byte elements
gbconv_status_t launch_transpose_b(const void *in, void *out, long long B, int R, int Cn,
                                   int elem_bytes, cudaStream_t st);
// scale = gamma / sqrt(var + eps), shift = bn_beta + (bias - mean) * scale
gbconv_status_t launch_bn_fold(int K, const float *gamma, const float *bn_beta, const float *mean,
                               const float *var, float eps, const float *bias, float *scale,
                               float *shift, cudaStream_t st);
// zeroes dx at rows u*h' + a, columns v*w' + b (NHWC, out_dtype of d)
gbconv_status_t launch_zero_phase(const Dims &d, void *dx, int a, int b, cudaStream_t st);
// out[i] = y[i] > 0 ? g[i] : 0 (F32/BF16 each; out may alias g when the types match)
gbconv_status_t launch_relu_grad(const void *y, int y_dtype, const void *g, int g_dtype, void *out,
                                 int out_dtype, long long n, cudaStream_t st);
// FFMA throughput of the current device (synchronous; CUDA events on st)
gbconv_status_t measure_ffma_rate(long long iters, double *tflops, cudaStream_t st);
gbconv_status_t launch_quantize_e4m3(const void *in, int in_dtype, long long rows, long long len,
                                     uint8_t *out, float *scale, cudaStream_t st);

// tc.cu: tensor-core (tcgen05) kernels.
struct TcConfig {
    int block_n;   // 32..256, multiple of 32
    int stages;
    int split_k;   // wgrad slices
    int raster;    // 0: output-channel tiles fastest
    int algo;      // GBCONV_ALGO_*
};
bool tc_fwd_supported(const Dims &d);
TcConfig tc_fwd_default_config(const Dims &d);
gbconv_status_t launch_tc_fwd(const Dims &d, const TcConfig &cfg, const void *x, const void *w,
                              const float *bias, const float *x_scale, const float *w_scale,
                              void *y, cudaStream_t st, const Fused &fz = Fused{});
// tc_fwd_shift.cu: stride-1 layers, one input band per channel block.
bool tc_fwd_shift_supported(const Dims &d, int block_n);
bool tc_fwd_shift_preferred(const Dims &d, int block_n);  // automatic choice
gbconv_status_t launch_tc_fwd_shift(const Dims &d, const TcConfig &cfg, const void *x,
                                    const void *w, const float *bias, const float *x_scale,
                                    const float *w_scale, void *y, cudaStream_t st,
                                    const Fused &fz = Fused{});
// tc_fwd_t.cu: band kernel with output channels on the MMA's M (strides by
// phase decomposition; 1x1 stride-1 layers as a flat GEMM), and the data
// gradient of strided layers by sub-pixel phases on the same kernel.
bool tc_dgrad_t_supported(const Dims &d);
gbconv_status_t launch_tc_dgrad_t(const Dims &d, const void *dy, const void *wT, void *dx,
                                  cudaStream_t st);
int tc_fwd_t_tile(const Dims &d);  // output-channel tile (64 / 128), 0 if unsuitable
gbconv_status_t launch_tc_fwd_t(const Dims &d, const void *x, const void *w, const float *bias,
                                const float *x_scale, const float *w_scale, void *y,
                                cudaStream_t st, const Fused &fz = Fused{});
// tc_fwd_p.cu: pixel-major band kernel (BF16, multi-tap, K <= 128, strides up
// to 4 by phases, resident filter) on one SM (form 1) or a pair of SMs (form 2).
// tc_fwd_p_form: the form it would take (want 1 or 2: only that form; 0: the
// automatic choice), 0 when it cannot take the layer.
int tc_fwd_p_form(const Dims &d, int want);
gbconv_status_t launch_tc_fwd_p(const Dims &d, int form, const void *x, const void *w,
                                const float *bias, void *y, cudaStream_t st);
gbconv_status_t launch_tc_grouped(int count, const Dims *d, const TcConfig *cfg,
                                  const void *const *x, const void *const *w,
                                  const float *const *bias, void *const *y, cudaStream_t st);
bool tc_wgrad_supported(const Dims &d);
long long tc_wgrad_pixel_steps(const Dims &d);  // 64-pixel reduction steps
TcConfig tc_wgrad_default_config(const Dims &d);
gbconv_status_t launch_tc_wgrad_partials(const Dims &d, const TcConfig &cfg, const void *x,
                                         const void *g, float *ws, cudaStream_t st);
// tc_wgrad_shift.cu: stride-1 multi-tap layers, the taps of one filter row as
// row shifts of one input band (reduction steps = bands of output rows).
bool tc_wgrad_shift_supported(const Dims &d);
long long tc_wgrad_shift_bands(const Dims &d);
int tc_wgrad_shift_default_slices(const Dims &d);
gbconv_status_t launch_tc_wgrad_shift_partials(const Dims &d, int slices, const void *x,
                                               const void *g, float *ws, cudaStream_t st);

// tmap.cpp: tensor-map encoding through the driver entry points.
gbconv_status_t encode_im2col_act(CUtensorMap *m, const Dims &d, const void *x, int elem_bytes,
                                  int channels_per_pixel, int pixels_per_column);
// Tiled map; elem_strides (may be null = all 1) is the traversal step per
// dimension: a box of b elements with step t loads ceil(b / t) of them.
gbconv_status_t encode_tiled(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *ptr,
                             const uint64_t *dims, const uint64_t *strides_bytes,
                             const uint32_t *box, CUtensorMapSwizzle swz,
                             const uint32_t *elem_strides = nullptr);

}  // namespace gbc
