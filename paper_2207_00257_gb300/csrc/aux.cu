// aux.cu -- small memory-bound kernels around the convolutions:
//   * fixed-order compensated (Neumaier) sum of split-K slices (weight gradient),
//   * bias gradient db[k] = sum_{n,p,q} g[n,k,p,q] (paper Sec. 5.B backward pass),
//   * 180-degree filter rotation with C and K exchanged (data gradient as a
//     forward convolution),
//   * FP8 E4M3 operand preparation: per-group scale max|v|/448 and RNE
//     quantisation with saturation.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"

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
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float sum = 0.f, comp = 0.f;
        for (int s = 0; s < slices; ++s) neumaier(sum, comp, ws[(long long)s * n + i]);
        out[i] = sum + comp;
    }
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// NHWC: g is [M][K]; block y = slice of rows, threads stride over k.
template <typename T>
__global__ void bias_grad_nhwc(const T *__restrict__ g, long long M, int K, int slices,
                               float *__restrict__ part) {
    long long r0 = M * blockIdx.y / slices, r1 = M * (blockIdx.y + 1) / slices;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        float sum = 0.f, comp = 0.f;
        for (long long r = r0; r < r1; ++r) neumaier(sum, comp, to_f(g[r * K + k]));
        part[(long long)blockIdx.y * K + k] = sum + comp;
    }
}

// NCHW: g is [N][K][P*Q]; block (k, slice over n) reduces its rows with a
// fixed-shape tree, then writes one partial.
template <typename T>
__global__ void bias_grad_nchw(const T *__restrict__ g, int N, int K, long long PQ, int slices,
                               float *__restrict__ part) {
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

// amax per group into amax_bits[r] (non-negative floats order like their bits).
template <typename T>
__global__ void amax_kernel(const T *__restrict__ in, long long len, unsigned *__restrict__ amax_bits) {
    __shared__ float sh[256];
    const long long base = (long long)blockIdx.y * len;
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(to_f(in[base + i])));
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

template <typename T>
__global__ void quant_kernel(const T *__restrict__ in, long long len,
                             const unsigned *__restrict__ amax_bits, uint8_t *__restrict__ out) {
    const long long base = (long long)blockIdx.y * len;
    const float s = scale_of(amax_bits[blockIdx.y]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        float q = __fdiv_rn(to_f(in[base + i]), s);
        out[base + i] = (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    }
}

__global__ void finalize_scale(unsigned *__restrict__ amax_bits, long long rows) {
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
    reduce_slices_kernel<<<grid_for(n, 256), 256, 0, st>>>(ws, slices, n, out);
    return cuda_status(cudaGetLastError());
}

gbconv_status_t launch_bias_grad(const Dims &d, const void *g, float *db, float *ws, int slices,
                                 cudaStream_t st) {
    if (d.layout == GBCONV_NHWC) {
        dim3 grid((unsigned)((d.K + 255) / 256), (unsigned)slices);
        if (d.in_dtype == GBCONV_F32)
            bias_grad_nhwc<float><<<grid, 256, 0, st>>>((const float *)g, d.M(), d.K, slices, ws);
        else
            bias_grad_nhwc<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)g, d.M(),
                                                                d.K, slices, ws);
    } else {
        dim3 grid((unsigned)d.K, (unsigned)slices);
        long long PQ = (long long)d.P * d.Q;
        if (d.in_dtype == GBCONV_F32)
            bias_grad_nchw<float><<<grid, 256, 0, st>>>((const float *)g, d.N, d.K, PQ, slices, ws);
        else
            bias_grad_nchw<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)g, d.N, d.K,
                                                                PQ, slices, ws);
    }
    gbconv_status_t s = cuda_status(cudaGetLastError());
    if (s != GBCONV_OK) return s;
    return launch_reduce_slices(ws, slices, d.K, db, st);
}

gbconv_status_t launch_rotate_filter(const Dims &d, const void *w, void *w_rot, cudaStream_t st) {
    long long total = (long long)d.K * d.R * d.S * d.C;
    unsigned g = grid_for(total, 256);
    if (d.in_dtype == GBCONV_BF16)
        rotate_krsc<__nv_bfloat16><<<g, 256, 0, st>>>((const __nv_bfloat16 *)w,
                                                      (__nv_bfloat16 *)w_rot, d.K, d.R, d.S, d.C);
    else if (d.in_dtype == GBCONV_F32)
        rotate_krsc<float><<<g, 256, 0, st>>>((const float *)w, (float *)w_rot, d.K, d.R, d.S, d.C);
    else
        return GBCONV_ERR_UNSUPPORTED;
    return cuda_status(cudaGetLastError());
}

gbconv_status_t launch_quantize_e4m3(const void *in, int in_dtype, long long rows, long long len,
                                     uint8_t *out, float *scale, cudaStream_t st) {
    if (rows > 65535) return GBCONV_ERR_UNSUPPORTED;
    unsigned *amax = reinterpret_cast<unsigned *>(scale);
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float) * rows, st);
    if (e != cudaSuccess) return cuda_status(e);
    long long per = (len + 255) / 256;
    unsigned gx = (unsigned)(per < 1 ? 1 : per);
    unsigned cap = (unsigned)((sm_count() * 8 + rows - 1) / rows);
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    dim3 grid(gx, (unsigned)rows);
    if (in_dtype == GBCONV_F32) {
        amax_kernel<float><<<grid, 256, 0, st>>>((const float *)in, len, amax);
        quant_kernel<float><<<grid, 256, 0, st>>>((const float *)in, len, amax, out);
    } else if (in_dtype == GBCONV_BF16) {
        amax_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)in, len, amax);
        quant_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)in, len, amax, out);
    } else {
        return GBCONV_ERR_UNSUPPORTED;
    }
    finalize_scale<<<grid_for(rows, 256), 256, 0, st>>>(amax, rows);
    return cuda_status(cudaGetLastError());
}

}  // namespace gbc
