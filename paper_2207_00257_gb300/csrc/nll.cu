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
// Gradient: one write per element of [N][C]: -w_n * g at (n, target[n]) of
// counted rows (g = grad_out[n], grad_out[0], or grad_out[0] / total_weight),
// zero elsewhere.
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

__global__ void nll_grad(const float *__restrict__ grad_out, const int64_t *__restrict__ target,
                         const float *__restrict__ weight, long long N, long long C,
                         long long ignore_index, int reduction,
                         const float *__restrict__ total_weight, float *grad_in, unsigned *err) {
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const long long total = N * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long n = i / C, c = i - n * C;
        const long long t = target[n];
        float v = 0.f;
        if (t == c && t != ignore_index) {
            const float w = weight ? weight[t] : 1.f;
            const float g = reduction == 0 ? grad_out[n]
                            : reduction == 1 ? grad_out[0] / total_weight[0] : grad_out[0];
            v = -w * g;
        } else if (c == 0 && t != ignore_index && (t < 0 || t >= C)) {
            atomicOr(err, DEVERR_BAD_INDEX);
        }
        grad_in[i] = v;
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
    const long long total = N * C;
    if (total == 0) return GBCONV_OK;
    const long long blocks = (total + 255) / 256;
    const unsigned grid = (unsigned)(blocks < (long long)sm_count() * 8 ? blocks : sm_count() * 8);
    return cuda_status(launch_pdl(nll_grad, dim3(grid), dim3(256), 0, st, grad_out, target, weight,
                                  N, C, ignore_index, reduction, total_weight, grad_in, g.err));
}

}  // namespace gbc
