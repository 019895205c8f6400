// nll.cu -- negative log-likelihood loss, forward and gradient (the
// ClassNLLCriterion updateOutput / updateGradInput kernels that ResNet-50
// training runs after the network, paper Sec. 5.B, whose block reduction
// synchronises with __syncthreads).
//
// logp [N][C] fp32, target [N] int64, optional class weights [C]. Row n counts
// with weight w_n = weight[target[n]] unless target[n] == ignore_index:
//   none: out[n] = -w_n * logp[n][target[n]];  sum: out = sum_n (.);
//   mean: out = sum_n (.) / sum_n w_n;  total_weight = sum_n w_n.
// Forward: deterministic two-pass reduction. Pass 1 gives each block a fixed
// range of NLL_ROWS rows (4 per thread, then a shared-memory tree with
// __syncthreads), so the partial sums depend only on N; pass 2 (one block)
// reduces the partials in the same fixed tree order. A target outside
// [0, C) that is not ignore_index sets DEVERR_BAD_INDEX in the device error
// word and counts as ignored.
// Gradient: one write per element of [N][C], a warp per row: -w_n * g at
// (n, target[n]) of counted rows (g = grad_out[n], grad_out[0], or
// grad_out[0] / total_weight), zero elsewhere.
#include <cstdint>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int NLL_THREADS = 256;
constexpr int NLL_ROWS = 4 * NLL_THREADS;  // rows per block of pass 1

// Fixed-order tree sum of one value per thread (blockDim.x == NLL_THREADS).
__device__ __forceinline__ float block_sum(float v, float *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = NLL_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const float r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(NLL_THREADS) nll_partials(const float *__restrict__ logp,
                                                             const int64_t *__restrict__ target,
                                                             const float *__restrict__ weight,
                                                             long long N, long long C,
                                                             long long ignore_index, int reduction,
                                                             float *out, float *partials,
                                                             unsigned *err) {
    __shared__ float sh[NLL_THREADS];
    ptx::griddep_wait();
    float loss = 0.f, wsum = 0.f;
    const long long r0 = (long long)blockIdx.x * NLL_ROWS;
#pragma unroll
    for (int i = 0; i < NLL_ROWS / NLL_THREADS; ++i) {
        const long long n = r0 + i * NLL_THREADS + threadIdx.x;
        if (n >= N) break;
        const long long t = target[n];
        float v = 0.f;
        if (t != ignore_index) {
            if (t < 0 || t >= C) {
                atomicOr(err, DEVERR_BAD_INDEX);
            } else {
                const float w = weight ? weight[t] : 1.f;
                v = -w * logp[n * C + t];
                loss += v;
                wsum += w;
            }
        }
        if (reduction == 0) out[n] = v;
    }
    loss = block_sum(loss, sh);
    wsum = block_sum(wsum, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = loss;
        partials[2 * blockIdx.x + 1] = wsum;
        ptx::griddep_launch();
    }
}

__global__ void __launch_bounds__(NLL_THREADS) nll_final(const float *__restrict__ partials,
                                                          int nb, int reduction, float *out,
                                                          float *total_weight) {
    __shared__ float sh[NLL_THREADS];
    ptx::griddep_wait();
    // each thread sums its fixed stride of blocks in order, then the fixed tree
    float loss = 0.f, wsum = 0.f;
    for (int b = threadIdx.x; b < nb; b += NLL_THREADS) {
        loss += partials[2 * b];
        wsum += partials[2 * b + 1];
    }
    loss = block_sum(loss, sh);
    wsum = block_sum(wsum, sh);
    if (threadIdx.x == 0) {
        if (reduction == 1) out[0] = loss / wsum;
        if (reduction == 2) out[0] = loss;
        *total_weight = wsum;
        ptx::griddep_launch();
    }
}

// One row per warp-iteration: the row's zeros (16-byte stores when C % 4 == 0
// and grad_in is 16-byte aligned) with -w_n * g at column target[n].
__global__ void nll_grad(const float *__restrict__ grad_out, const int64_t *__restrict__ target,
                         const float *__restrict__ weight, long long N, long long C,
                         long long ignore_index, int reduction,
                         const float *__restrict__ total_weight, float *grad_in, int vec4,
                         unsigned *err) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long n = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); n < N;
         n += warps) {
        const long long t = target[n];
        long long tc = -1;  // column of the row's only non-zero
        float v = 0.f;
        if (t != ignore_index) {
            if (t < 0 || t >= C) {
                if (lane == 0) atomicOr(err, DEVERR_BAD_INDEX);
            } else {
                const float w = weight ? weight[t] : 1.f;
                const float g = reduction == 0 ? grad_out[n]
                                : reduction == 1 ? grad_out[0] / total_weight[0] : grad_out[0];
                v = -w * g;
                tc = t;
            }
        }
        float *row = grad_in + n * C;
        if (vec4) {
            for (long long c = 4 * lane; c < C; c += 128) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tc >= c && tc < c + 4) {
                    const int k = (int)(tc - c);
                    q.x = k == 0 ? v : 0.f;
                    q.y = k == 1 ? v : 0.f;
                    q.z = k == 2 ? v : 0.f;
                    q.w = k == 3 ? v : 0.f;
                }
                *reinterpret_cast<float4 *>(row + c) = q;
            }
        } else {
            for (long long c = lane; c < C; c += 32) row[c] = c == tc ? v : 0.f;
        }
    }
}

}  // namespace

size_t nll_workspace_bytes(long long N) {
    const long long nb = (N + NLL_ROWS - 1) / NLL_ROWS;
    return (size_t)(nb > 0 ? nb : 1) * 2 * sizeof(float);
}

gbconv_status_t launch_nll_fwd(const float *logp, const int64_t *target, const float *weight,
                               long long N, long long C, long long ignore_index, int reduction,
                               float *out, float *total_weight, float *ws, cudaStream_t st) {
    const Guard g = make_guard();
    if (!g.err) return GBCONV_ERR_CUDA;
    const long long nb = (N + NLL_ROWS - 1) / NLL_ROWS;
    if (nb > 0) {
        cudaError_t e = launch_pdl(nll_partials, dim3((unsigned)nb), dim3(NLL_THREADS), 0, st, logp,
                                   target, weight, N, C, ignore_index, reduction, out, ws, g.err);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(launch_pdl(nll_final, dim3(1), dim3(NLL_THREADS), 0, st,
                                  (const float *)ws, (int)nb, reduction, out, total_weight));
}

gbconv_status_t launch_nll_grad(const float *grad_out, const int64_t *target, const float *weight,
                                long long N, long long C, long long ignore_index, int reduction,
                                const float *total_weight, float *grad_in, cudaStream_t st) {
    const Guard g = make_guard();
    if (!g.err) return GBCONV_ERR_CUDA;
    if (N * C == 0) return GBCONV_OK;
    const int vec4 = C % 4 == 0 && reinterpret_cast<uintptr_t>(grad_in) % 16 == 0;
    const long long blocks = (N + 7) / 8;  // 8 rows (warps) per block
    const unsigned grid = (unsigned)(blocks < (long long)sm_count() * 16 ? blocks : sm_count() * 16);
    return cuda_status(launch_pdl(nll_grad, dim3(grid), dim3(256), 0, st, grad_out, target, weight,
                                  N, C, ignore_index, reduction, total_weight, grad_in, vec4,
                                  g.err));
}

}  // namespace gbc
