// aux.cu -- small memory-bound kernels around the convolutions:
//   * fixed-order compensated (Neumaier) sum of split-K slices (weight gradient),
//   * bias gradient db[k] = sum_{n,p,q} g[n,k,p,q] (paper Sec. 5.B backward pass),
//   * 180-degree filter rotation with C and K exchanged (data gradient as a
//     forward convolution),
//   * FP8 E4M3 operand preparation: per-group scale max|v|/448 and RNE
//     quantisation with saturation,
//   * the gradient through the ReLU that follows a convolution (the upstream
//     gradient masked where the forward output is not positive).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

// Neumaier's compensated summation step: sum + v with the rounding error of
// the addition collected in comp.
__device__ __forceinline__ void neumaier(float &sum, float &comp, float v) {
    float t = sum + v;
    if (fabsf(sum) >= fabsf(v))
        comp += (sum - t) + v;
    else
        comp += (v - t) + sum;
    sum = t;
}

__global__ void reduce_slices_kernel(const float *__restrict__ ws, int slices, long long n,
                                     float *__restrict__ out) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float sum = 0.f, comp = 0.f;
        int s = 0;
        for (; s + 8 <= slices; s += 8) {  // eight loads in flight, summed in slice order
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = ws[(long long)(s + j) * n + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) neumaier(sum, comp, v[j]);
        }
        for (; s < slices; ++s) neumaier(sum, comp, ws[(long long)s * n + i]);
        out[i] = sum + comp;
    }
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// NHWC: g is [M][K]. Block (x, y) sums the 32 channels k = 32x + lane over
// the rows of slice y; its 8 warps take interleaved rows (row = r0 + warp +
// 8i), each with a compensated running sum, then a fixed-shape tree joins the
// 8 warp sums. Loads are 64-byte coalesced runs along k.
template <typename T>
__global__ void __launch_bounds__(256) bias_grad_nhwc(const T *__restrict__ g, long long M, int K,
                                                      int slices, float *__restrict__ part) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    __shared__ float sh[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const long long r0 = M * blockIdx.y / slices, r1 = M * (blockIdx.y + 1) / slices;
    float sum = 0.f, comp = 0.f;
    if (k < K) {
        long long r = r0 + wid;
        for (; r + 24 < r1; r += 32) {  // four independent loads in flight
            const float a = to_f(g[r * K + k]), b = to_f(g[(r + 8) * K + k]);
            const float c = to_f(g[(r + 16) * K + k]), e = to_f(g[(r + 24) * K + k]);
            neumaier(sum, comp, a);
            neumaier(sum, comp, b);
            neumaier(sum, comp, c);
            neumaier(sum, comp, e);
        }
        for (; r < r1; r += 8) neumaier(sum, comp, to_f(g[r * K + k]));
    }
    sh[wid][lane] = sum + comp;
    __syncthreads();
    if (wid == 0 && k < K) {
        float a = (sh[0][lane] + sh[1][lane]) + (sh[2][lane] + sh[3][lane]);
        float b = (sh[4][lane] + sh[5][lane]) + (sh[6][lane] + sh[7][lane]);
        part[(long long)blockIdx.y * K + k] = a + b;
    }
}

// NHWC BF16 with K a power of two from 8 to 4096: thread t owns the
// channel octet o = t % (K/8) (one 16-byte load per row) and the rows
// r0 + t/(K/8) + i*(512/(K/8)) of block y's slice, eight loads in flight,
// eight compensated running sums; the block then joins the row phases of
// each channel in fixed order. The 64-byte warp loads of bias_grad_nhwc kept
// too few bytes in flight to stream the tensor.
__device__ __forceinline__ void widen_bf16x2(uint32_t v, float &lo, float &hi) {
    lo = __uint_as_float(v << 16);
    hi = __uint_as_float(v & 0xffff0000u);
}

__global__ void __launch_bounds__(512) bias_grad_nhwc_bf16x8(const __nv_bfloat16 *__restrict__ g,
                                                              long long M, int K, int slices,
                                                              float *__restrict__ part) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    constexpr int UNROLL = 8;
    __shared__ float sh[512 * 8];  // [row phase][K]: 512/(K/8) x K floats
    const int oct = K >> 3;
    const int o = threadIdx.x % oct, rp = threadIdx.x / oct, rstep = 512 / oct;
    const long long r0 = M * blockIdx.x / slices, r1 = M * (blockIdx.x + 1) / slices;
    float sum[8], comp[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) sum[e] = comp[e] = 0.f;
    const uint4 *gv = reinterpret_cast<const uint4 *>(g);
    auto add = [&](const uint4 &v) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float lo, hi;
            widen_bf16x2(w[i], lo, hi);
            neumaier(sum[2 * i], comp[2 * i], lo);
            neumaier(sum[2 * i + 1], comp[2 * i + 1], hi);
        }
    };
    long long r = r0 + rp;
    for (; r + (long long)(UNROLL - 1) * rstep < r1; r += (long long)UNROLL * rstep) {
        uint4 v[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) v[u] = __ldg(gv + (r + (long long)u * rstep) * oct + o);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) add(v[u]);
    }
    for (; r < r1; r += rstep) add(__ldg(gv + r * oct + o));
#pragma unroll
    for (int e = 0; e < 8; ++e) sh[rp * K + o * 8 + e] = sum[e] + comp[e];
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += 512) {
        float s2 = 0.f, c2 = 0.f;
        for (int p = 0; p < rstep; ++p) neumaier(s2, c2, sh[p * K + k]);
        part[(long long)blockIdx.x * K + k] = s2 + c2;
    }
}

// out[i] = sum over slices of ws[s][i] for a short vector (one warp per
// output): lanes take slices lane, lane + 32, ... with compensated sums, then
// a fixed-shape shuffle tree.
__global__ void reduce_slices_warp(const float *__restrict__ ws, int slices, int n,
                                   float *__restrict__ out) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;  // whole warps
    float sum = 0.f, comp = 0.f;
    int s = lane;
    for (; s + 7 * 32 < slices; s += 8 * 32) {  // eight loads in flight, summed in slice order
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = ws[(long long)(s + 32 * j) * n + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) neumaier(sum, comp, v[j]);
    }
    for (; s < slices; s += 32) neumaier(sum, comp, ws[(long long)s * n + i]);
    float t = sum + comp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) out[i] = t;
}

// NCHW: g is [N][K][P*Q]; block (k, slice over n) reduces its rows with a
// fixed-shape tree, then writes one partial.
template <typename T>
__global__ void bias_grad_nchw(const T *__restrict__ g, int N, int K, long long PQ, int slices,
                               float *__restrict__ part) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    __shared__ float sh[256];
    const int k = blockIdx.x;
    int n0 = (int)((long long)N * blockIdx.y / slices), n1 = (int)((long long)N * (blockIdx.y + 1) / slices);
    float sum = 0.f, comp = 0.f;
    for (int n = n0; n < n1; ++n) {
        const T *row = g + ((long long)n * K + k) * PQ;
        for (long long i = threadIdx.x; i < PQ; i += blockDim.x) neumaier(sum, comp, to_f(row[i]));
    }
    sh[threadIdx.x] = sum + comp;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.y * K + k] = sh[0];
}

// w [K][R][S][C] -> w_rot [C][R][S][K] with w_rot[c][r][s][k] = w[k][R-1-r][S-1-s][c]
template <typename T>
__global__ void rotate_krsc(const T *__restrict__ w, T *__restrict__ wr, int K, int R, int S,
                            int C) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    long long total = (long long)K * R * S * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        // i indexes the output [c][r][s][k]
        int k = (int)(i % K);
        long long t = i / K;
        int s = (int)(t % S);
        t /= S;
        int r = (int)(t % R);
        int c = (int)(t / R);
        wr[i] = w[(((long long)k * R + (R - 1 - r)) * S + (S - 1 - s)) * C + c];
    }
}

// Filter transpose w[k][r][s][c] -> wT[c][r][s][k] (no rotation): the filter
// of the sub-pixel data-gradient phases.
template <typename T>
__global__ void transpose_krsc(const T *__restrict__ w, T *__restrict__ wt, int K, int RS, int C) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    long long total = (long long)K * RS * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        // i indexes the output [c][t][k]
        int k = (int)(i % K);
        long long t = i / K;
        int rs = (int)(t % RS);
        int c = (int)(t / RS);
        wt[i] = w[((long long)k * RS + rs) * C + c];
    }
}

// Batched transpose out[b][j][i] = in[b][i][j] (in: [B][R][Cn]) through 32x32
// shared-memory tiles (one padding column against bank conflicts): the NCHW
// <-> NHWC and KCRS -> KRSC layout transforms around the NHWC tensor-core path.
template <typename T>
__global__ void transpose_b(const T *__restrict__ in, T *__restrict__ out, int R, int Cn) {
    __shared__ T tile[32][33];
    ptx::griddep_wait();
    if (threadIdx.x == 0 && threadIdx.y == 0) ptx::griddep_launch();
    const long long b = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const T *src = in + b * (long long)R * Cn;
    T *dst = out + b * (long long)R * Cn;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, j = j0 + threadIdx.x;
        if (i < R && j < Cn) tile[k][threadIdx.x] = src[(long long)i * Cn + j];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int j = j0 + k, i = i0 + threadIdx.x;
        if (i < R && j < Cn) dst[(long long)j * R + i] = tile[threadIdx.x][k];
    }
}

// Inference batch normalisation after a convolution with bias, folded into
// the fused forward's per-channel scale and shift (sqrtf and the division
// are the correctly rounded FP32 operations).
__global__ void bn_fold_kernel(int K, const float *__restrict__ gamma,
                               const float *__restrict__ bn_beta, const float *__restrict__ mean,
                               const float *__restrict__ var, float eps,
                               const float *__restrict__ bias, float *__restrict__ scale,
                               float *__restrict__ shift) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float a = gamma[k] / sqrtf(var[k] + eps);
    scale[k] = a;
    shift[k] = bn_beta[k] + ((bias ? bias[k] : 0.f) - mean[k]) * a;
}

// Zeroes the positions (n, u*h' + a, v*w' + b, :) of an NHWC tensor: a
// sub-pixel phase of the data gradient that no filter tap reaches.
template <typename T>
__global__ void zero_phase(T *__restrict__ dx, int N, int H, int W, int C, int u, int v, int a,
                           int b) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const int Ha = (H - a + u - 1) / u, Wb = (W - b + v - 1) / v;
    const long long total = (long long)N * Ha * Wb * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long t = i / C;
        const int wq = (int)(t % Wb);
        t /= Wb;
        const int hq = (int)(t % Ha);
        const int n = (int)(t / Ha);
        dx[(((long long)n * H + (long long)hq * u + a) * W + (long long)wq * v + b) * C + c] = T(0.f);
    }
}

// Vector of 8 consecutive input values as float (16 B of BF16, or two 16-B
// loads of FP32). The caller guarantees alignment and bounds.
__device__ __forceinline__ void load8(const float *p, float (&v)[8]) {
    float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16 *p, float (&v)[8]) {
    uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// amax per group into amax_bits[r] (non-negative floats order like their
// bits). VEC: 8 values per thread step (requires len % 8 == 0 and 16-byte
// aligned groups), else one value per step.
template <typename T, bool VEC>
__global__ void amax_kernel(const T *__restrict__ in, long long len, unsigned *__restrict__ amax_bits) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    __shared__ float sh[256];
    const T *g = in + (long long)blockIdx.y * len;
    float m = 0.f;
    if (VEC) {
        constexpr int U = 4;  // four 8-element steps in flight per thread
        const long long stride = (long long)gridDim.x * blockDim.x * 8;
        long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 8;
        for (; i + (U - 1) * stride < len; i += U * stride) {
            float v[U][8];
#pragma unroll
            for (int u = 0; u < U; ++u) load8(g + i + u * stride, v[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int k = 0; k < 8; ++k) m = fmaxf(m, fabsf(v[u][k]));
        }
        for (; i < len; i += stride) {
            float v[8];
            load8(g + i, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) m = fmaxf(m, fabsf(v[k]));
        }
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
             i += (long long)gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf(to_f(g[i])));
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(amax_bits + blockIdx.y, __float_as_uint(sh[0]));
}

__device__ __forceinline__ float scale_of(unsigned amax_bits) {
    float s = __fdiv_rn(__uint_as_float(amax_bits), 448.0f);
    return (s >= 1.0e-12f) ? s : 1.0e-12f;
}

// v / s rounded to nearest even in binary32, for a normal s > 0 and its
// correctly rounded reciprocal r, by multiplication and exact remainders:
//  1. q0 = v*r, then one Markstein refinement q1 = q0 + (v - s*q0)*r (both
//     fused), which leaves q1 a faithful rounding of v/s;
//  2. for a faithful q1 the remainder e = v - s*q1 is exactly representable
//     (Boldo and Daumas, representable correcting terms), so one more fused
//     step gives it exactly;
//  3. v/s lies between q1 and its neighbour q2 on e's side; it passes their
//     midpoint iff |e| > s*|q2 - q1|/2, where the right side is exact (a power
//     of two times s). Equality is a tie: the even significand wins.
// Exactness needs s*|q2 - q1|/2 normal: every quotient at or above 2^-10 in
// magnitude (where E4M3 rounding decisions happen, s >= 1e-12) has it; below,
// q may differ from the rounded quotient, but both round to E4M3 zero.
__device__ __forceinline__ float div_rn_by_recip(float v, float s, float r) {
    const float q0 = v * r;
    const float q1 = fmaf(fmaf(-q0, s, v), r, q0);
    const float e = fmaf(-q1, s, v);
    if (e == 0.f || q1 == 0.f || !isfinite(q1)) return q1;
    // neighbour of q1 towards the exact quotient (e and q1 of equal sign: away from zero)
    const int step = (e > 0.f) == (q1 > 0.f) ? 1 : -1;
    const float q2 = __int_as_float(__float_as_int(q1) + step);
    const float half = s * (fabsf(q2 - q1) * 0.5f);
    const float ae = fabsf(e);
    if (ae < half) return q1;
    if (ae > half) return q2;
    return (__float_as_int(q1) & 1) ? q2 : q1;
}

__device__ __forceinline__ uint8_t e4m3_of(float v, float s, float r) {
    return (uint8_t)__nv_cvt_float_to_fp8(div_rn_by_recip(v, s, r), __NV_SATFINITE, __NV_E4M3);
}

template <typename T, bool VEC>
__global__ void quant_kernel(const T *__restrict__ in, long long len,
                             const unsigned *__restrict__ amax_bits, uint8_t *__restrict__ out) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const long long base = (long long)blockIdx.y * len;
    const float s = scale_of(amax_bits[blockIdx.y]);
    const float r = __frcp_rn(s);
    if (VEC) {
        // four 8-element steps per trip, all loads issued before the divisions,
        // so that the memory latency overlaps the arithmetic
        constexpr int U = 4;
        const long long stride = (long long)gridDim.x * blockDim.x * 8;
        long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 8;
        for (; i + (U - 1) * stride < len; i += U * stride) {
            float v[U][8];
#pragma unroll
            for (int u = 0; u < U; ++u) load8(in + base + i + u * stride, v[u]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t lo = 0, hi = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    lo |= (uint32_t)e4m3_of(v[u][k], s, r) << (8 * k);
                    hi |= (uint32_t)e4m3_of(v[u][4 + k], s, r) << (8 * k);
                }
                *reinterpret_cast<uint2 *>(out + base + i + u * stride) = make_uint2(lo, hi);
            }
        }
        for (; i < len; i += stride) {
            float v[8];
            load8(in + base + i, v);
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lo |= (uint32_t)e4m3_of(v[k], s, r) << (8 * k);
                hi |= (uint32_t)e4m3_of(v[4 + k], s, r) << (8 * k);
            }
            *reinterpret_cast<uint2 *>(out + base + i) = make_uint2(lo, hi);
        }
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
             i += (long long)gridDim.x * blockDim.x)
            out[base + i] = e4m3_of(to_f(in[base + i]), s, r);
    }
}

// Gradient through ReLU: out[i] = y[i] > 0 ? g[i] : 0, converted to the
// output type (BF16 by round to nearest even). VEC: 8 elements per step with
// 16-byte accesses (n % 8 == 0, every pointer 16-byte aligned).
__device__ __forceinline__ void store8(float *p, const float (&v)[8]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store8(__nv_bfloat16 *p, const float (&v)[8]) {
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = u;
}
template <typename TO>
__device__ __forceinline__ TO from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename TY, typename TG, typename TO, bool VEC>
__global__ void relu_grad_kernel(const TY *__restrict__ y, const TG *g, TO *out, long long n) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const long long step = (long long)gridDim.x * blockDim.x;
    if (VEC) {
        for (long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 8; i < n; i += step * 8) {
            float vy[8], vg[8];
            load8(y + i, vy);
            load8(g + i, vg);
#pragma unroll
            for (int k = 0; k < 8; ++k) vg[k] = vy[k] > 0.f ? vg[k] : 0.f;
            store8(out + i, vg);
        }
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += step)
            out[i] = from_f<TO>(to_f(y[i]) > 0.f ? to_f(g[i]) : 0.f);
    }
}

// FFMA issue-rate probe: 8 independent fused multiply-add chains per thread,
// 16 steps each per loop trip (the multiplier and addend come from the caller,
// so nothing folds). The result is written only if it equals a value no chain
// reaches, which keeps every chain live.
__global__ void __launch_bounds__(256) ffma_rate_kernel(long long iters, float m, float c,
                                                        float *out) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], m, c);
    }
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += a[j];
    if (t == -1.2345e30f) out[0] = t;
}

__global__ void finalize_scale(unsigned *__restrict__ amax_bits, long long rows) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        float s = scale_of(amax_bits[r]);
        amax_bits[r] = __float_as_uint(s);
    }
}

unsigned grid_for(long long n, int block, int per_sm = 8) {
    long long g = (n + block - 1) / block;
    long long cap = (long long)sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

gbconv_status_t launch_reduce_slices(const float *ws, int slices, long long n, float *out,
                                     cudaStream_t st) {
    if (n <= 0) return GBCONV_OK;
    return cuda_status(
        launch_pdl(reduce_slices_kernel, dim3(grid_for(n, 256)), dim3(256), 0, st, ws, slices, n, out));
}

gbconv_status_t launch_bias_grad(const Dims &d, const void *g, float *db, float *ws, int slices,
                                 cudaStream_t st) {
    cudaError_t e;
    const bool pow2 = d.K >= 8 && d.K <= 4096 && (d.K & (d.K - 1)) == 0;
    if (d.layout == GBCONV_NHWC && d.in_dtype == GBCONV_BF16 && pow2 &&
        (reinterpret_cast<uintptr_t>(g) & 15) == 0) {
        e = launch_pdl(bias_grad_nhwc_bf16x8, dim3((unsigned)slices), dim3(512), 0, st,
                       (const __nv_bfloat16 *)g, d.M(), d.K, slices, ws);
        if (e != cudaSuccess) return cuda_status(e);
        return cuda_status(launch_pdl(reduce_slices_warp, dim3((unsigned)((d.K + 7) / 8)), dim3(256), 0,
                                      st, (const float *)ws, slices, d.K, db));
    }
    slices = std::min(slices, 128);  // the generic kernels: at most 128 row slices
    if (d.layout == GBCONV_NHWC) {
        dim3 grid((unsigned)((d.K + 31) / 32), (unsigned)slices);
        if (d.in_dtype == GBCONV_F32)
            e = launch_pdl(bias_grad_nhwc<float>, grid, dim3(256), 0, st, (const float *)g, d.M(), d.K,
                           slices, ws);
        else
            e = launch_pdl(bias_grad_nhwc<__nv_bfloat16>, grid, dim3(256), 0, st,
                           (const __nv_bfloat16 *)g, d.M(), d.K, slices, ws);
    } else {
        dim3 grid((unsigned)d.K, (unsigned)slices);
        long long PQ = (long long)d.P * d.Q;
        if (d.in_dtype == GBCONV_F32)
            e = launch_pdl(bias_grad_nchw<float>, grid, dim3(256), 0, st, (const float *)g, d.N, d.K,
                           PQ, slices, ws);
        else
            e = launch_pdl(bias_grad_nchw<__nv_bfloat16>, grid, dim3(256), 0, st,
                           (const __nv_bfloat16 *)g, d.N, d.K, PQ, slices, ws);
    }
    if (e != cudaSuccess) return cuda_status(e);
    return launch_reduce_slices(ws, slices, d.K, db, st);
}

gbconv_status_t launch_rotate_filter(const Dims &d, const void *w, void *w_rot, cudaStream_t st) {
    long long total = (long long)d.K * d.R * d.S * d.C;
    unsigned g = grid_for(total, 256);
    cudaError_t e;
    if (d.in_dtype == GBCONV_BF16)
        e = launch_pdl(rotate_krsc<__nv_bfloat16>, dim3(g), dim3(256), 0, st,
                       (const __nv_bfloat16 *)w, (__nv_bfloat16 *)w_rot, d.K, d.R, d.S, d.C);
    else if (d.in_dtype == GBCONV_F32)
        e = launch_pdl(rotate_krsc<float>, dim3(g), dim3(256), 0, st, (const float *)w,
                       (float *)w_rot, d.K, d.R, d.S, d.C);
    else
        return GBCONV_ERR_UNSUPPORTED;
    return cuda_status(e);
}

gbconv_status_t launch_transpose_filter(const Dims &d, const void *w, void *wt, cudaStream_t st) {
    long long total = (long long)d.K * d.R * d.S * d.C;
    unsigned g = grid_for(total, 256);
    if (d.in_dtype != GBCONV_BF16) return GBCONV_ERR_UNSUPPORTED;
    return cuda_status(launch_pdl(transpose_krsc<__nv_bfloat16>, dim3(g), dim3(256), 0, st,
                                  (const __nv_bfloat16 *)w, (__nv_bfloat16 *)wt, d.K, d.R * d.S,
                                  d.C));
}

gbconv_status_t launch_transpose_b(const void *in, void *out, long long B, int R, int Cn,
                                   int elem_bytes, cudaStream_t st) {
    if (B == 0 || R == 0 || Cn == 0) return GBCONV_OK;
    if (B > 65535 || (R + 31) / 32 > 65535) return GBCONV_ERR_UNSUPPORTED;
    const dim3 grid((unsigned)((Cn + 31) / 32), (unsigned)((R + 31) / 32), (unsigned)B);
    const dim3 block(32, 8);
    cudaError_t e;
    if (elem_bytes == 2)
        e = launch_pdl(transpose_b<uint16_t>, grid, block, 0, st, (const uint16_t *)in,
                       (uint16_t *)out, R, Cn);
    else
        e = launch_pdl(transpose_b<uint32_t>, grid, block, 0, st, (const uint32_t *)in,
                       (uint32_t *)out, R, Cn);
    return cuda_status(e);
}

gbconv_status_t launch_bn_fold(int K, const float *gamma, const float *bn_beta, const float *mean,
                               const float *var, float eps, const float *bias, float *scale,
                               float *shift, cudaStream_t st) {
    return cuda_status(launch_pdl(bn_fold_kernel, dim3((K + 255) / 256), dim3(256), 0, st, K, gamma,
                                  bn_beta, mean, var, eps, bias, scale, shift));
}

gbconv_status_t launch_zero_phase(const Dims &d, void *dx, int a, int b, cudaStream_t st) {
    const int Ha = (d.H - a + d.u - 1) / d.u, Wb = (d.W - b + d.v - 1) / d.v;
    long long total = (long long)d.N * Ha * Wb * d.C;
    if (total <= 0) return GBCONV_OK;
    unsigned g = grid_for(total, 256);
    cudaError_t e;
    if (d.out_dtype == GBCONV_F32)
        e = launch_pdl(zero_phase<float>, dim3(g), dim3(256), 0, st, (float *)dx, d.N, d.H, d.W,
                       d.C, d.u, d.v, a, b);
    else
        e = launch_pdl(zero_phase<__nv_bfloat16>, dim3(g), dim3(256), 0, st, (__nv_bfloat16 *)dx,
                       d.N, d.H, d.W, d.C, d.u, d.v, a, b);
    return cuda_status(e);
}

gbconv_status_t launch_quantize_e4m3(const void *in, int in_dtype, long long rows, long long len,
                                     uint8_t *out, float *scale, cudaStream_t st) {
    if (rows > 65535) return GBCONV_ERR_UNSUPPORTED;
    unsigned *amax = reinterpret_cast<unsigned *>(scale);
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float) * rows, st);
    if (e != cudaSuccess) return cuda_status(e);
    const int eb = in_dtype == GBCONV_F32 ? 4 : 2;
    const bool vec = len % 8 == 0 && (reinterpret_cast<uintptr_t>(in) % 16) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) % 8) == 0 && (len * eb) % 16 == 0;
    const long long per = vec ? (len / 8 + 255) / 256 : (len + 255) / 256;
    unsigned gx = (unsigned)(per < 1 ? 1 : per);
    unsigned cap = (unsigned)((sm_count() * 8 + rows - 1) / rows);
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    dim3 grid(gx, (unsigned)rows);
#define GBC_QUANT(T, V)                                                                  \
    do {                                                                               \
        e = launch_pdl(amax_kernel<T, V>, grid, dim3(256), 0, st, (const T *)in, len, amax); \
        if (e == cudaSuccess)                                                          \
            e = launch_pdl(quant_kernel<T, V>, grid, dim3(256), 0, st, (const T *)in, len, \
                           (const unsigned *)amax, out);                               \
    } while (0)
    if (in_dtype == GBCONV_F32) {
        if (vec) GBC_QUANT(float, true); else GBC_QUANT(float, false);
    } else if (in_dtype == GBCONV_BF16) {
        if (vec) GBC_QUANT(__nv_bfloat16, true); else GBC_QUANT(__nv_bfloat16, false);
    } else {
        return GBCONV_ERR_UNSUPPORTED;
    }
#undef GBC_QUANT
    if (e == cudaSuccess)
        e = launch_pdl(finalize_scale, dim3(grid_for(rows, 256)), dim3(256), 0, st, amax, rows);
    return cuda_status(e);
}


gbconv_status_t launch_relu_grad(const void *y, int y_dtype, const void *g, int g_dtype, void *out,
                                 int out_dtype, long long n, cudaStream_t st) {
    if (n <= 0) return GBCONV_OK;
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec = n % 8 == 0 && al(y) && al(g) && al(out);
    const unsigned grid = grid_for(vec ? n / 8 : n, 256);
    cudaError_t e = cudaErrorInvalidValue;
#define GBC_RG(TY, TG, TO)                                                                          \
    e = vec ? launch_pdl(relu_grad_kernel<TY, TG, TO, true>, dim3(grid), dim3(256), 0, st,          \
                         (const TY *)y, (const TG *)g, (TO *)out, n)                                \
            : launch_pdl(relu_grad_kernel<TY, TG, TO, false>, dim3(grid), dim3(256), 0, st,         \
                         (const TY *)y, (const TG *)g, (TO *)out, n)
    const int code = (y_dtype == GBCONV_BF16) * 4 + (g_dtype == GBCONV_BF16) * 2 + (out_dtype == GBCONV_BF16);
    switch (code) {
        case 0: GBC_RG(float, float, float); break;
        case 1: GBC_RG(float, float, __nv_bfloat16); break;
        case 2: GBC_RG(float, __nv_bfloat16, float); break;
        case 3: GBC_RG(float, __nv_bfloat16, __nv_bfloat16); break;
        case 4: GBC_RG(__nv_bfloat16, float, float); break;
        case 5: GBC_RG(__nv_bfloat16, float, __nv_bfloat16); break;
        case 6: GBC_RG(__nv_bfloat16, __nv_bfloat16, float); break;
        default: GBC_RG(__nv_bfloat16, __nv_bfloat16, __nv_bfloat16); break;
    }
#undef GBC_RG
    return cuda_status(e);
}


gbconv_status_t measure_ffma_rate(long long iters, double *tflops, cudaStream_t st) {
    const int blocks = sm_count() * 4, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBCONV_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBCONV_ERR_CUDA;
    }
    float *sink = nullptr;  // never written (see the kernel)
    ffma_rate_kernel<<<blocks, threads, 0, st>>>(iters / 8 + 1, 0.9999999f, 1e-7f, sink);  // warm-up
    cudaEventRecord(e0, st);
    ffma_rate_kernel<<<blocks, threads, 0, st>>>(iters, 0.9999999f, 1e-7f, sink);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return GBCONV_ERR_CUDA;
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return GBCONV_OK;
}

}  // namespace gbc
