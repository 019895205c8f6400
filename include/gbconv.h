/*
 * gbconv.h -- C ABI of a GB300 (sm_103a) dense 2D convolution library.
 *
 * The operation is the convolution that the paper (arXiv 2207.00257) names as
 * the critical kernel of its PyTorch case: Sec. 1 and Sec. 5.A (PyTorch's
 * native CPU backend computes 2D convolution as six nested loops) and Sec. 5.B
 * (the forward and backward passes of ResNet-50's convolutional layers, done
 * there as im2col + GEMM on NCHW tensors). With stride (u, v), zero padding
 * (ph, pw) and dilation (dh, dw):
 *
 *   P = floor((H + 2*ph - dh*(R-1) - 1) / u) + 1,  Q likewise with W, pw, dw, S, v
 *   y[n,k,p,q] = b[k] + sum_{c,r,s} x[n,c, p*u + r*dh - ph, q*v + s*dw - pw] * w[k,c,r,s]
 *
 * (cross-correlation; x outside the image reads as 0), optionally followed by
 * ReLU. For the loss L = sum g*y the backward entry points compute
 *
 *   dx[n,c,h,w] = sum over (k,r,s,p,q) with p*u+r*dh-ph = h, q*v+s*dw-pw = w of g[n,k,p,q]*w[k,c,r,s]
 *   dw[k,c,r,s] = sum_{n,p,q} g[n,k,p,q] * x[n,c,p*u+r*dh-ph, q*v+s*dw-pw]
 *   db[k]       = sum_{n,p,q} g[n,k,p,q]
 *
 * Layouts. GBCONV_NHWC: x[n][h][w][c], filters w[k][r][s][c] (KRSC), y and g
 * y[n][p][q][k]. GBCONV_NCHW: x[n][c][h][w], filters w[k][c][r][s] (KCRS), y and
 * g y[n][k][p][q]. All tensors are dense and contiguous in that order.
 *
 * Ownership. The caller owns every tensor and every workspace; all tensor and
 * workspace pointers are DEVICE pointers unless a comment says "host". The
 * library owns only small host-side caches (tensor maps, tuning table) and one
 * static device error word. No entry point allocates device memory.
 *
 * Asynchrony and errors. Compute entry points validate their arguments on the
 * host, enqueue work on `stream` and return without synchronising. Their
 * status covers validation and launch errors only: on any error nothing is
 * launched. Every wait inside a kernel is bounded; a wait that runs out sets
 * the device error word and the kernel exits early. gbconv_get_device_error()
 * synchronises the stream and reports (and clears) that word. Entry points are
 * thread-safe (caches are mutex-guarded); calls that overlap on the GPU and
 * write the same output or workspace race, as with any CUDA kernel.
 */
#ifndef GBCONV_H
#define GBCONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBCONV_OK = 0,
    GBCONV_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, bad enum, P or Q < 1 */
    GBCONV_ERR_UNSUPPORTED = 2,   /* valid convolution this entry point does not implement */
    GBCONV_ERR_ALIGNMENT = 3,     /* channel count or pointer misses the 16-byte rule of TMA */
    GBCONV_ERR_WORKSPACE = 4,     /* workspace smaller than gbconv_workspace_size() */
    GBCONV_ERR_CUDA = 5,          /* a CUDA runtime or driver call failed */
    GBCONV_ERR_TIMEOUT = 6        /* a bounded in-kernel wait ran out */
} gbconv_status_t;

typedef enum { GBCONV_F32 = 0, GBCONV_BF16 = 1, GBCONV_E4M3 = 2 } gbconv_dtype_t;
typedef enum { GBCONV_NCHW = 0, GBCONV_NHWC = 1 } gbconv_layout_t;
/* GBCONV_OP_GROUPED: one problem as the body of conv2d_grouped runs it (its
 * tuning-table entry holds the problem's tile width in the grouped launch). */
typedef enum {
    GBCONV_OP_FWD = 0,
    GBCONV_OP_DGRAD = 1,
    GBCONV_OP_WGRAD = 2,
    GBCONV_OP_GROUPED = 3
} gbconv_op_t;

#define GBCONV_FLAG_BIAS 1u   /* add b[k] (fp32 for F32 output, else fp32 as well) */
#define GBCONV_FLAG_RELU 2u   /* y = max(y, 0) after the bias */

/* One convolution. Sizes are element counts. in_dtype is the type of x and w
 * (and of g for the backward entry points); out_dtype is the type of y (or
 * dx). Supported combinations:
 *   F32  -> F32   NCHW or NHWC, any stride/pad/dilation (CUDA-core FFMA kernel)
 *   BF16 -> BF16 or F32   NHWC, C % 8 == 0, K % 8 == 0 (tensor cores, FP32 accumulate);
 *                 the forward also takes BF16 NCHW (x [N,C,H,W], w [K,C,R,S], y
 *                 [N,K,P,Q]): transpose kernels bring x and w to NHWC/KRSC in the
 *                 workspace, the NHWC path runs, and y is transposed back
 *                 (gbconv_workspace_size(GBCONV_OP_FWD) gives the bytes)
 *   E4M3 -> BF16  NHWC, C % 16 == 0, K % 8 == 0 (tensor cores, FP32 accumulate,
 *                 y = b + x_scale * w_scale[k] * sum(xq * wq))
 * Padding must be in [0, 127] and dilation*(R-1) <= 127 (the im2col TMA range).
 * N may be 0 (an empty batch): conv2d_fwd and conv2d_dgrad then do nothing
 * (tensor pointers may be NULL) and conv2d_wgrad writes zeros to dw and db.
 *
 * Channel groups (groups = G > 1; G = C = K is the depthwise convolution):
 * C and K must be multiples of G; output channel k of group g = k / (K/G)
 * reads input channels g*C/G .. g*C/G + C/G - 1, and w holds C/G channels
 * per output channel: [K,R,S,C/G] (NHWC) or [K,C/G,R,S] (NCHW). The forward
 * (conv2d_fwd, conv2d_fwd_fused) supports groups: BF16/E4M3 NHWC with C/G
 * and K/G multiples of 8 (16 for E4M3) runs each group on the tensor cores
 * in one persistent launch; depthwise NHWC (C/G = K/G = 1, C % 8 == 0) runs a
 * CUDA-core kernel with 16-byte channel vectors; the rest (F32/BF16 in) runs
 * the CUDA-core implicit GEMM per group. conv2d_dgrad and conv2d_wgrad (and
 * conv2d_dgrad_noalloc) take groups on the CUDA-core kernels (FP32
 * accumulation, one grid layer per group); conv2d_grouped returns
 * GBCONV_ERR_UNSUPPORTED for G > 1. */
typedef struct {
    int32_t N, C, H, W, K, R, S;
    int32_t stride_h, stride_w;
    int32_t pad_h, pad_w;
    int32_t dil_h, dil_w;
    int32_t in_dtype;   /* gbconv_dtype_t */
    int32_t out_dtype;  /* gbconv_dtype_t */
    int32_t layout;     /* gbconv_layout_t */
    uint32_t flags;     /* GBCONV_FLAG_* */
    int32_t groups;     /* channel groups G (0 or 1: none); see below */
} gbconv_problem_t;

/* Launch configuration of one convolution (chosen by the autotuner or set by
 * hand). block_n: output-channel tile (32..256, tensor-core paths) ; stages:
 * shared-memory pipeline depth; split_k: number of slices the reduction is
 * cut into (wgrad); raster: 0 = output-channel tiles fastest, 1 = pixel tiles
 * fastest; algo (tensor-core forward and data gradient): GBCONV_ALGO_AUTO,
 * GBCONV_ALGO_IM2COL (one TMA im2col tile per filter tap),
 * GBCONV_ALGO_SHIFT (stride 1 only: one input band per channel block, filter
 * taps as row shifts of it) or GBCONV_ALGO_SHIFT_T (the same band with the
 * GEMM transposed: output channels on the MMA's M, 256 positions on N; stride
 * 1 and K <= 128 only), GBCONV_ALGO_SIMT (the CUDA-core FFMA kernel, for
 * F32 and BF16 inputs; a reference point for the tensor-core paths),
 * GBCONV_ALGO_PBAND (BF16 multi-tap layers with K <= 128, strides up to 4:
 * output pixels on the MMA's M, one input band per stride phase and channel
 * block, the filter resident in shared memory, one SM per 128-position tile)
 * or GBCONV_ALGO_PBAND_PAIR (the same on pairs of SMs: one 256-row MMA per
 * pair, each SM holding half of the filter). For the weight gradient (BF16
 * NHWC, C % 64 == 0): GBCONV_ALGO_AUTO / GBCONV_ALGO_IM2COL (one work unit per
 * filter tap, dy and an im2col tile of x loaded per tap), GBCONV_ALGO_SHIFT
 * (stride 1, multi-tap: one unit per filter row, dy and one x band loaded per
 * row and the row's taps read as shifts of the band, a third of the
 * shared-memory ingest for 3x3 layers) or GBCONV_ALGO_SIMT (CUDA cores). A
 * zero field means "library default". */
#define GBCONV_ALGO_AUTO 0
#define GBCONV_ALGO_IM2COL 1
#define GBCONV_ALGO_SHIFT 2
#define GBCONV_ALGO_SHIFT_T 3
#define GBCONV_ALGO_SIMT 4
#define GBCONV_ALGO_PBAND 5
#define GBCONV_ALGO_PBAND_PAIR 6
typedef struct {
    int32_t block_n;
    int32_t stages;
    int32_t split_k;
    int32_t raster;
    int32_t algo;
} gbconv_config_t;

/* A CUDA stream (cudaStream_t). NULL means the legacy default stream. */
typedef void *gbconv_stream_t;

/* Output spatial size P, Q of the formula above. Host only, no GPU use.
 * Returns GBCONV_ERR_INVALID_ARG for invalid problems (P or Q < 1, sizes < 1,
 * negative padding, stride or dilation < 1). */
gbconv_status_t gbconv_output_dims(const gbconv_problem_t *prob, int32_t *P, int32_t *Q);

/* Bytes of device workspace `op` needs for `prob` (0 when none). Host only.
 * FWD: 0. DGRAD: the filter rotated by 180 degrees with C and K exchanged
 * (tensor-core path, stride 1), rounded up to 256 bytes; 0 otherwise.
 * WGRAD: (split_k * K*R*S*C/G + 304 * K) fp32 partial sums (weight slices
 * and 304 bias slices), rounded up to 256 bytes. */
gbconv_status_t gbconv_workspace_size(int32_t op, const gbconv_problem_t *prob, size_t *bytes);

/* Forward convolution (paper Sec. 5.B, forward pass of a convolutional layer).
 *   x [N,H,W,C] (NHWC) or [N,C,H,W] (NCHW), in_dtype
 *   w [K,R,S,C] (NHWC) or [K,C,R,S] (NCHW), in_dtype
 *   bias [K] fp32, read when GBCONV_FLAG_BIAS is set (may be NULL otherwise)
 *   x_scale: device pointer to one fp32 (E4M3 only, else ignored)
 *   w_scale: device pointer to K fp32 (E4M3 only, else ignored)
 *   y [N,P,Q,K] (NHWC) or [N,K,P,Q] (NCHW), out_dtype; must not alias x or w
 *   ws / ws_bytes: workspace: gbconv_workspace_size(GBCONV_OP_FWD) bytes, 16-byte
 *                  aligned (only BF16 NCHW needs any; else may be NULL / 0)
 * Tensor-core paths require x, w, y 16-byte aligned. */
gbconv_status_t conv2d_fwd(const gbconv_problem_t *prob, const void *x, const void *w,
                           const float *bias, const float *x_scale, const float *w_scale,
                           void *y, void *ws, size_t ws_bytes, gbconv_stream_t stream);

/* Forward with the layers that follow a ResNet-50 convolution fused into the
 * epilogue (paper Sec. 5.B: the model's convolutions are followed by batch
 * normalisation and tensor additions):
 *
 *   y[n,p,q,k] = act(scale[k] * conv(x, w)[n,p,q,k] + bias[k] + residual[n,p,q,k])
 *
 * conv(x, w) is the convolution of conv2d_fwd without its bias (for E4M3
 * inputs already multiplied by x_scale * w_scale[k]); act is ReLU when
 * GBCONV_FLAG_RELU is set. Inference batch normalisation folds into (scale,
 * bias): see gbconv_bn_fold.
 *   prob, x, w, x_scale, w_scale, y, ws, ws_bytes, stream: as in conv2d_fwd
 *   bias     [K] fp32, read when GBCONV_FLAG_BIAS is set (the shift)
 *   scale    [K] fp32 device pointer, or NULL for 1
 *   residual y's shape, layout and out_dtype, or NULL for 0. It may be y
 *            itself (in-place add: each element is read before it is
 *            written, by the same thread) but not x or w. Tensor-core paths
 *            require it 16-byte aligned (else GBCONV_ERR_ALIGNMENT).
 * Arithmetic: FP32, in the order scale, bias, residual, activation, then one
 * rounding to out_dtype. Not available through conv2d_grouped. */
gbconv_status_t conv2d_fwd_fused(const gbconv_problem_t *prob, const void *x, const void *w,
                                 const float *bias, const float *scale, const void *residual,
                                 const float *x_scale, const float *w_scale, void *y, void *ws,
                                 size_t ws_bytes, gbconv_stream_t stream);

/* Inference batch normalisation of a convolution with bias b, folded into
 * conv2d_fwd_fused's per-channel scale and shift (paper Sec. 5.B, the batch
 * normalisation layers of ResNet-50):
 *   scale[k] = gamma[k] / sqrt(var[k] + eps)
 *   shift[k] = bn_beta[k] + (b[k] - mean[k]) * scale[k]
 * All arrays are K fp32 device pointers; bias may be NULL (b = 0). FP32 with
 * correctly rounded square root and division. Asynchronous on stream;
 * GBCONV_ERR_INVALID_ARG for K < 0, a NULL required pointer or eps < 0 (or NaN). */
gbconv_status_t gbconv_bn_fold(int32_t K, const float *gamma, const float *bn_beta,
                               const float *mean, const float *var, float eps, const float *bias,
                               float *scale, float *shift, gbconv_stream_t stream);

/* Negative log-likelihood loss (paper Sec. 5.B: ClassNLLCriterion_updateOutput
 * and _updateGradInput, the custom CUDA kernels ResNet-50 training runs after
 * the network; their block reduction synchronises with __syncthreads).
 *   logp [N][C] fp32 log-probabilities; target [N] int64 class indices;
 *   weight [C] fp32 class weights or NULL (all 1); rows whose target equals
 *   ignore_index count with weight 0. w_n = weight[target[n]] for the others.
 *   reduction 0 (none): out[n] = -w_n * logp[n][target[n]]  (out holds N floats)
 *   reduction 2 (sum):  out[0] = sum_n -w_n * logp[n][target[n]]
 *   reduction 1 (mean): out[0] = (that sum) / sum_n w_n   (NaN when every row is ignored)
 *   total_weight[0] = sum_n w_n (all reductions; the gradient of mean needs it).
 * All pointers are device pointers. The forward is a deterministic two-pass
 * FP32 reduction (fixed row blocks, fixed tree order) and needs
 * gbconv_nll_workspace_size(N) bytes of workspace. A target outside [0, C)
 * that is not ignore_index counts as ignored and makes the next
 * gbconv_get_device_error return GBCONV_ERR_INVALID_ARG. */
gbconv_status_t gbconv_nll_workspace_size(int64_t N, size_t *bytes);
gbconv_status_t gbconv_nll_loss_fwd(const float *logp, const int64_t *target, const float *weight,
                                    int64_t N, int64_t C, int64_t ignore_index, int32_t reduction,
                                    float *out, float *total_weight, void *ws, size_t ws_bytes,
                                    gbconv_stream_t stream);
/* Gradient of the loss with respect to logp, written to every element of
 * grad_in [N][C]: -w_n * g at (n, target[n]) of counted rows, 0 elsewhere, with
 * g = grad_out[n] (none), grad_out[0] (sum) or grad_out[0] / total_weight[0]
 * (mean; total_weight from the forward). */
gbconv_status_t gbconv_nll_loss_bwd(const float *grad_out, const int64_t *target,
                                    const float *weight, int64_t N, int64_t C,
                                    int64_t ignore_index, int32_t reduction,
                                    const float *total_weight, float *grad_in,
                                    gbconv_stream_t stream);

/* Data gradient (paper Sec. 5.B, backward pass; the transposed convolution).
 *   dy [N,P,Q,K] or [N,K,P,Q] (in_dtype), w as in conv2d_fwd (in_dtype),
 *   dx [N,H,W,C] or [N,C,H,W] (out_dtype). dx is fully overwritten.
 * BF16 NHWC with stride 1 and pad <= dil*(R-1) runs on the tensor cores as a
 * forward convolution of dy with the rotated filter. Other BF16 NHWC layers
 * (strides up to 4, any padding, channels multiples of 8) run on the tensor
 * cores by sub-pixel phases: for each output phase (h mod u, w mod v) the
 * taps that reach it form a stride-1 correlation of dy with the transposed
 * filter, written to every u-th row and v-th column of dx; phases no tap
 * reaches are zeroed. Both tensor-core forms need the workspace (the filter,
 * rotated or transposed: K*R*S*C*2 bytes, see gbconv_workspace_size).
 * Everything else runs on a CUDA-core gather kernel with FP32 accumulation. */
gbconv_status_t conv2d_dgrad(const gbconv_problem_t *prob, const void *dy, const void *w,
                             void *dx, void *ws, size_t ws_bytes, gbconv_stream_t stream);

/* Weight and bias gradient (paper Sec. 5.B, backward pass).
 *   x as in conv2d_fwd, dy as in conv2d_dgrad (both in_dtype)
 *   dw [K,R,S,C] or [K,C,R,S] fp32, fully overwritten
 *   db [K] fp32 or NULL (then not computed)
 * The reduction over N*P*Q is cut into split_k slices whose fp32 partial sums
 * go to the workspace; a second kernel adds the slices in a fixed order with
 * compensated (Neumaier) summation, so results are deterministic. */
gbconv_status_t conv2d_wgrad(const gbconv_problem_t *prob, const void *x, const void *dy,
                             float *dw, float *db, void *ws, size_t ws_bytes,
                             gbconv_stream_t stream);

/* Many independent forward convolutions in ONE persistent launch.
 *   probs: HOST array of `count` problems (1 <= count <= 64 per launch; larger
 *          counts are split into launches of 64), all BF16 -> BF16 NHWC.
 *   x, w, bias, y: HOST arrays of `count` DEVICE pointers (bias entries may be
 *          NULL when the problem has no GBCONV_FLAG_BIAS).
 * All per-problem descriptors travel as kernel parameters, so the call makes
 * no host-to-device copy and can be captured in a CUDA graph. Tile configs
 * come from the tuning table (gbconv_tune) or the built-in heuristic. */
gbconv_status_t conv2d_grouped(int32_t count, const gbconv_problem_t *probs,
                               const void *const *x, const void *const *w,
                               const float *const *bias, void *const *y, void *ws,
                               size_t ws_bytes, gbconv_stream_t stream);

/* Gradient through the ReLU of a forward run with GBCONV_FLAG_RELU (paper
 * Sec. 5.B, backward pass: every ResNet-50 convolution is followed by a
 * rectifier, whose derivative masks the upstream gradient):
 *   g_out[i] = y[i] > 0 ? g[i] : 0      for 0 <= i < n
 * y is the forward's output (y = max(z, 0), so y > 0 exactly where z > 0),
 * g the upstream gradient of y, g_out the gradient of z, ready for
 * conv2d_dgrad / conv2d_wgrad. Element types y_dtype, g_dtype, out_dtype are
 * GBCONV_F32 or GBCONV_BF16 each (else GBCONV_ERR_UNSUPPORTED); a BF16 output
 * is rounded to nearest even. All three are device pointers to n elements in
 * any common layout. g_out may be g itself (same dtype; in place) but must not
 * overlap y or partly overlap g (GBCONV_ERR_INVALID_ARG). n = 0 does nothing.
 * Asynchronous on stream; no workspace. */
gbconv_status_t gbconv_relu_grad(const void *y, int32_t y_dtype, const void *g, int32_t g_dtype,
                                 void *g_out, int32_t out_dtype, int64_t n, gbconv_stream_t stream);

/* FP8 operand preparation for the E4M3 forward path. `in` holds `rows`
 * contiguous groups of `len` values (in_dtype F32 or BF16). Per group,
 * entirely in binary32:
 *   scale[r] = max(max_i |in[r,i]| / 448, 1e-12)
 *   out[r,i] = E4M3(in[r,i] / scale[r]), round to nearest even, saturating to +-448
 * rows = 1 gives the per-tensor activation scale; rows = K over a KRSC filter
 * gives per-output-channel weight scales. out (uint8 codes) and scale are
 * device pointers; no workspace. */
gbconv_status_t gbconv_quantize_e4m3(const void *in, int32_t in_dtype, int64_t rows, int64_t len,
                                     uint8_t *out, float *scale, gbconv_stream_t stream);

/* Tuning. gbconv_get_config returns the config `op` would use for `prob`
 * (tuned entry if present, else the heuristic); gbconv_set_config stores one.
 * gbconv_tune times every candidate config on the caller's buffers (same
 * arguments as the op: FWD a=x, b=w, out=y; DGRAD a=dy, b=w, out=dx; WGRAD
 * a=x, b=dy, out=dw; GROUPED as FWD, timing the grouped launch's body on this
 * one problem at every tile width, BF16 NHWC only) with `reps` launches each
 * on `stream`, stores and returns the fastest. The table is keyed by problem,
 * op and device name and can be saved to / loaded from a JSON file (host
 * path). conv2d_grouped takes each problem's GROUPED entry when there is one,
 * else the forward heuristic. */
gbconv_status_t gbconv_get_config(int32_t op, const gbconv_problem_t *prob, gbconv_config_t *cfg);
gbconv_status_t gbconv_set_config(int32_t op, const gbconv_problem_t *prob,
                                  const gbconv_config_t *cfg);
gbconv_status_t gbconv_tune(int32_t op, const gbconv_problem_t *prob, const void *a,
                            const void *b, const float *bias, void *out, void *ws,
                            size_t ws_bytes, int32_t reps, gbconv_stream_t stream,
                            gbconv_config_t *best);
gbconv_status_t gbconv_tune_cache_save(const char *path);
gbconv_status_t gbconv_tune_cache_load(const char *path);

/* Synchronises `stream`, then returns GBCONV_ERR_TIMEOUT if a bounded wait in
 * any kernel ran out since the last call (and clears the word), GBCONV_ERR_CUDA
 * if the synchronisation failed, else GBCONV_OK. */
gbconv_status_t gbconv_get_device_error(gbconv_stream_t stream);

/* Static, human-readable name of a status. Never NULL. */
const char *gbconv_status_string(gbconv_status_t status);

/* Test and diagnosis controls (not needed in normal use):
 *   GBCONV_DEBUG_WAIT_LIMIT_NS: time limit of every in-kernel wait (default
 *       2e9 ns; 0 restores the default);
 *   GBCONV_DEBUG_SKIP_LOADS: when 1, tensor-core kernels issue no loads, so
 *       their consumers' waits run out and the kernel reports a timeout. */
#define GBCONV_DEBUG_WAIT_LIMIT_NS 1
#define GBCONV_DEBUG_SKIP_LOADS 2
gbconv_status_t gbconv_debug_set(int32_t key, int64_t value);

/* Data gradient that allocates nothing, for callers that cannot call
 * cudaMalloc or hand the library a workspace: code running under a framework
 * whose own allocator must own every device byte, code with a device-memory
 * budget fixed at start-up, and code that enqueues work where an allocation
 * would stall or be refused. The paper has no counterpart: it is a packaging
 * variant of conv2d_dgrad, not part of the method.
 *
 * Same arguments, layouts and results as conv2d_dgrad minus the workspace.
 * Where conv2d_dgrad would place the rotated filter (BF16 NHWC, stride 1) or
 * the transposed filter (the sub-pixel phases of strided BF16 NHWC layers) in
 * the caller's workspace, this entry point uses a static device array of
 * GBCONV_DGRAD_STATIC_SCRATCH_BYTES bytes that the library holds on every GPU
 * that loads it, until the process exits. Filters whose K*R*S*C*2 bytes exceed
 * that size are refused with GBCONV_ERR_WORKSPACE before anything is enqueued.
 * Every other problem runs here on the CUDA-core kernel and needs no scratch
 * at all (as does a problem whose stored config asks for GBCONV_ALGO_SIMT).
 *
 * The first call on each device looks up the array's device address (a CUDA
 * runtime query, done once per device with that device current); make that
 * first call before capturing a stream. Every call on a device shares the one
 * array and overwrites all of the scratch it reads, so no clearing is needed,
 * but calls that overlap on the same GPU (other streams, other host threads)
 * race on it: serialise them. */
#define GBCONV_DGRAD_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u)
gbconv_status_t conv2d_dgrad_noalloc(const gbconv_problem_t *prob, const void *dy,
                                     const void *w, void *dx, gbconv_stream_t stream);

/* Measured FP32 CUDA-core throughput of the current device, the roofline
 * denominator of the plain FP32 kernel (its nominal value is 2 x 128 FFMA
 * lanes x SMs x clock). Runs a probe kernel of fused multiply-adds (8
 * independent chains per thread, 4 blocks of 256 threads per SM, `iters`
 * trips of 128 FFMAs per thread) on `stream`, times it with CUDA events,
 * synchronises and writes TFLOP/s (2 flops per FFMA) to *tflops (host
 * pointer). Not for the hot path; the paper has no counterpart (it is part of
 * the measurement, not of the method). GBCONV_ERR_INVALID_ARG for iters < 1. */
gbconv_status_t gbconv_measure_ffma_tflops(int64_t iters, double *tflops, gbconv_stream_t stream);

/* Library version, as major*10000 + minor*100 + patch. */
int32_t gbconv_version(void);

/* Frees host-side caches (tensor maps, tuning table). Safe to call twice. */
void gbconv_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* GBCONV_H */
