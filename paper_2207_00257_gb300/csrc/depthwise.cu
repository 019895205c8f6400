// depthwise.cu -- forward of a convolution with small channel groups (C/G =
// K/G = CG in {1, 2, 4, 8}; CG = 1 is the depthwise convolution), NHWC, on
// the CUDA cores.
//
//   y[n,p,q,k] = act(alpha[k] * sum_{r,s,c<CG} x[n, p*u + r*dh - ph, q*v + s*dw - pw,
//                                                 g*CG + c] * w[k,r,s,c]
//                    + b[k] + z[n,p,q,k]),   g = k / CG
//
// (the forward of a convolutional layer, paper Sec. 5.B, with channel groups).
// With so few channels per group there is little reduction to share, so the
// layer is bound by memory traffic rather than tensor work. Because C/G = K/G,
// output channels k..k+7 (k a multiple of 8) read exactly input channels
// k..k+7: each thread owns 8 consecutive channels of PX consecutive output
// pixels of one row, reads x as 16-byte (BF16) or 32-byte (FP32) channel
// vectors per tap (a warp covers 32 x 8 consecutive channels, so its loads and
// stores are contiguous) and accumulates in FP32 in the order r, s, c. The
// filter is staged once per block in shared memory as FP32, laid out so that
// neighbouring lanes (neighbouring channel vectors) read neighbouring 16-byte
// words: [R*S][2*CG float4 slots][K/8 channel vectors].
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int DW_THREADS = 256;
constexpr int DW_SMEM_LIMIT = 200 * 1024;  // staged filter: R*S*K*CG fp32

struct DwParams {
    int N, C, H, W, P, Q, R, S, u, v, ph, pw, dh, dw;
    int relu;
    const float *bias, *alpha;
    const void *z;
};

__device__ __forceinline__ void load8(const float *p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16 *p, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
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

// Output pixels per thread (consecutive q), sharing each filter load (two for
// 8-channel groups, whose 64 weights per tap already fill the registers).
template <int CG>
struct Px {
    static constexpr int v = CG == 8 ? 2 : 4;
    static constexpr int min_blocks = 2;
};

// Raw 16-byte channel vector of 8 BF16 values, unpacked at use: all of a
// filter row's loads are issued before the first multiply.
__device__ __forceinline__ uint4 ldraw(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ void unpack8(const uint4 &u, float (&v)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// One tap's 8 x CG weights of channel vector cvi as 2*CG 16-byte shared
// loads, slot-major: a warp's lanes read consecutive words of one slot, with
// no bank conflict for any CG. Weight f of the vector (f = j*CG + c for
// output channel c0 + j and group channel c) is word f%4 of slot f/4.
template <int CG>
__device__ __forceinline__ void load_taps(const float4 *wp, int cv, float (&wv)[8 * CG]) {
#pragma unroll
    for (int i = 0; i < 2 * CG; ++i) {
        const float4 q = wp[i * cv];
        wv[4 * i] = q.x;
        wv[4 * i + 1] = q.y;
        wv[4 * i + 2] = q.z;
        wv[4 * i + 3] = q.w;
    }
}

// SC > 0 (BF16 input only): the filter width is the constant SC, so each
// filter row's SC x PX vector loads are unrolled and issued together. UNIT
// (horizontal stride and dilation 1): the PX pixels' SC taps cover only
// PX + SC - 1 input columns, each loaded (and, up to two channels per group,
// converted to FP32) once per filter row. Work items are numbered in 32 bits
// (fewer than 2^31, checked on the host).
template <typename Ti, typename To, int CG, int SC, bool UNIT>
__global__ void __launch_bounds__(DW_THREADS, Px<CG>::min_blocks) depthwise_kernel(
    const Ti *__restrict__ x, const Ti *__restrict__ w, To *y, const DwParams prm) {
    constexpr int PX = Px<CG>::v;
    extern __shared__ float4 wsm4[];  // [R*S][2*CG][C/8]
    float *wsm = reinterpret_cast<float *>(wsm4);
    const int RS = prm.R * prm.S, C = prm.C;  // C = K
    const int cv = C / 8;                     // channel vectors per pixel
    // The filter is a kernel input like x: read it after the dependency wait.
    ptx::griddep_wait();
    for (int i = threadIdx.x; i < RS * C * CG; i += blockDim.x) {
        const int e = i & 3;
        int t = i >> 2;
        const int cvi = t % cv;
        t /= cv;
        const int f = (t % (2 * CG)) * 4 + e, rs = t / (2 * CG);
        const int k = cvi * 8 + f / CG, c = f % CG;
        wsm[i] = static_cast<float>(w[((long long)k * RS + rs) * CG + c]);
    }
    __syncthreads();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const unsigned qb = (prm.Q + PX - 1) / PX;  // pixel blocks per output row
    const unsigned total = (unsigned)prm.N * prm.P * qb * cv;
    const To *z = static_cast<const To *>(prm.z);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c0 = (int)(i % (unsigned)cv) * 8;
        unsigned t = i / (unsigned)cv;
        const int q0 = (int)(t % qb) * PX;
        t /= qb;
        const int p = (int)(t % (unsigned)prm.P);
        const int n = (int)(t / (unsigned)prm.P);
        float acc[PX][8];
#pragma unroll
        for (int a = 0; a < PX; ++a)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[a][j] = 0.f;
        for (int r = 0; r < prm.R; ++r) {
            const int h = p * prm.u + r * prm.dh - prm.ph;
            if (h < 0 || h >= prm.H) continue;
            const Ti *xrow = x + ((long long)n * prm.H + h) * prm.W * C + c0;
            if constexpr (SC > 0 && UNIT) {
                constexpr int NX = PX + SC - 1;
                uint4 xr[NX];
#pragma unroll
                for (int e = 0; e < NX; ++e) {
                    const int ww = q0 + e - prm.pw;
                    xr[e] = (ww >= 0 && ww < prm.W) ? ldraw(xrow + ww * C) : make_uint4(0, 0, 0, 0);
                }
                if constexpr (CG <= 2) {
                    float xv[NX][8];
#pragma unroll
                    for (int e = 0; e < NX; ++e) unpack8(xr[e], xv[e]);
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        float wv[8 * CG];
                        load_taps<CG>(wsm4 + (r * SC + s) * 2 * CG * cv + c0 / 8, cv, wv);
#pragma unroll
                        for (int a = 0; a < PX; ++a)
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int gb = (j / CG) * CG;
#pragma unroll
                                for (int c = 0; c < CG; ++c)
                                    acc[a][j] = fmaf(xv[a + s][gb + c], wv[j * CG + c], acc[a][j]);
                            }
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        float wv[8 * CG];
                        load_taps<CG>(wsm4 + (r * SC + s) * 2 * CG * cv + c0 / 8, cv, wv);
#pragma unroll
                        for (int a = 0; a < PX; ++a) {
                            float xv[8];
                            unpack8(xr[a + s], xv);
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int gb = (j / CG) * CG;
#pragma unroll
                                for (int c = 0; c < CG; ++c)
                                    acc[a][j] = fmaf(xv[gb + c], wv[j * CG + c], acc[a][j]);
                            }
                        }
                    }
                }
                continue;
            } else if constexpr (SC > 0) {
                uint4 xr[SC][PX];
#pragma unroll
                for (int s = 0; s < SC; ++s)
#pragma unroll
                    for (int a = 0; a < PX; ++a) {
                        const int ww = (q0 + a) * prm.v + s * prm.dw - prm.pw;
                        xr[s][a] = (q0 + a < prm.Q && ww >= 0 && ww < prm.W)
                                       ? ldraw(xrow + (long long)ww * C)
                                       : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    float wv[8 * CG];
                    load_taps<CG>(wsm4 + (r * SC + s) * 2 * CG * cv + c0 / 8, cv, wv);
#pragma unroll
                    for (int a = 0; a < PX; ++a) {
                        float xv[8];
                        unpack8(xr[s][a], xv);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int gb = (j / CG) * CG;
#pragma unroll
                            for (int c = 0; c < CG; ++c)
                                acc[a][j] = fmaf(xv[gb + c], wv[j * CG + c], acc[a][j]);
                        }
                    }
                }
                continue;
            }
            for (int s = 0; s < prm.S; ++s) {
                // this tap's PX input vectors first (all loads in flight), then the math
                float xv[PX][8];
#pragma unroll
                for (int a = 0; a < PX; ++a) {
                    const int ww = (q0 + a) * prm.v + s * prm.dw - prm.pw;
                    if (q0 + a < prm.Q && ww >= 0 && ww < prm.W) {
                        load8(xrow + (long long)ww * C, xv[a]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) xv[a][j] = 0.f;
                    }
                }
                float wv[8 * CG];  // this tap's weights of the thread's 8 output channels
                load_taps<CG>(wsm4 + (r * prm.S + s) * 2 * CG * cv + c0 / 8, cv, wv);
#pragma unroll
                for (int a = 0; a < PX; ++a) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int gb = (j / CG) * CG;  // first channel of j's group in the vector
#pragma unroll
                        for (int c = 0; c < CG; ++c)
                            acc[a][j] = fmaf(xv[a][gb + c], wv[j * CG + c], acc[a][j]);
                    }
                }
            }
        }
#pragma unroll
        for (int a = 0; a < PX; ++a) {
            if (q0 + a >= prm.Q) break;
            const long long off = (((long long)n * prm.P + p) * prm.Q + q0 + a) * C + c0;
            float zv[8];
            if (z) load8(z + off, zv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float v = acc[a][j];
                if (prm.alpha) v = v * prm.alpha[c0 + j];
                if (prm.bias) v = prm.bias[c0 + j] + v;
                if (z) v = v + zv[j];
                if (prm.relu) v = fmaxf(v, 0.f);
                acc[a][j] = v;
            }
            store8(y + off, acc[a]);
        }
    }
}

template <typename Ti, typename To, int CG, int SC, bool UNIT = false>
gbconv_status_t launch_typed(const Dims &d, const void *x, const void *w, void *y, size_t smem,
                             const DwParams &prm, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(depthwise_kernel<Ti, To, CG, SC, UNIT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    constexpr int PX = Px<CG>::v;
    const long long total = (long long)d.N * d.P * ((d.Q + PX - 1) / PX) * (d.C / 8);
    const long long blocks = (total + DW_THREADS - 1) / DW_THREADS;
    const unsigned grid = (unsigned)std::min<long long>(blocks, (long long)sm_count() * 8);
    return cuda_status(launch_pdl(depthwise_kernel<Ti, To, CG, SC, UNIT>, dim3(grid), dim3(DW_THREADS), smem,
                                  st, static_cast<const Ti *>(x), static_cast<const Ti *>(w),
                                  static_cast<To *>(y), prm));
}

template <typename Ti, typename To>
gbconv_status_t launch_cg(const Dims &d, const void *x, const void *w, void *y, size_t smem,
                          const DwParams &prm, cudaStream_t st) {
    if constexpr (std::is_same<Ti, __nv_bfloat16>::value) {
        // unrolled rows where their registers fit: 1 or 2 channels per group, 4 for BF16 output
        const bool unit = d.v == 1 && d.dw == 1;
        if (d.S == 3 && d.C == d.G)
            return unit ? launch_typed<Ti, To, 1, 3, true>(d, x, w, y, smem, prm, st)
                        : launch_typed<Ti, To, 1, 3>(d, x, w, y, smem, prm, st);
        if (d.S == 3 && d.C == 2 * d.G)
            return unit ? launch_typed<Ti, To, 2, 3, true>(d, x, w, y, smem, prm, st)
                        : launch_typed<Ti, To, 2, 3>(d, x, w, y, smem, prm, st);
        if constexpr (std::is_same<To, __nv_bfloat16>::value) {
            if (d.S == 3 && d.C == 4 * d.G)
                return unit ? launch_typed<Ti, To, 4, 3, true>(d, x, w, y, smem, prm, st)
                            : launch_typed<Ti, To, 4, 3>(d, x, w, y, smem, prm, st);
        }
    }
    switch (d.C / d.G) {
        case 1: return launch_typed<Ti, To, 1, 0>(d, x, w, y, smem, prm, st);
        case 2: return launch_typed<Ti, To, 2, 0>(d, x, w, y, smem, prm, st);
        case 4: return launch_typed<Ti, To, 4, 0>(d, x, w, y, smem, prm, st);
        default: return launch_typed<Ti, To, 8, 0>(d, x, w, y, smem, prm, st);
    }
}

}  // namespace

bool depthwise_supported(const Dims &d) {
    if (d.G <= 1 || d.C != d.K || d.layout != GBCONV_NHWC || d.C % 8) return false;
    const int cg = d.C / d.G;  // = K / G
    if (cg != 1 && cg != 2 && cg != 4 && cg != 8) return false;
    if (!((d.in_dtype == GBCONV_F32 && d.out_dtype == GBCONV_F32) ||
          (d.in_dtype == GBCONV_BF16 && (d.out_dtype == GBCONV_BF16 || d.out_dtype == GBCONV_F32))))
        return false;
    // work items (at least two pixels each) are numbered in 32 bits
    if ((long long)d.N * d.P * ((d.Q + 1) / 2) * (d.C / 8) >= (1LL << 31)) return false;
    return (long long)d.R * d.S * d.C * cg * 4 <= DW_SMEM_LIMIT;
}

gbconv_status_t launch_depthwise(const Dims &d, const void *x, const void *w, const float *bias,
                                 void *y, cudaStream_t st, const Fused &fz) {
    if (!depthwise_supported(d)) return GBCONV_ERR_UNSUPPORTED;
    if (d.M() == 0) return GBCONV_OK;
    DwParams prm{d.N, d.C, d.H, d.W, d.P, d.Q, d.R, d.S, d.u, d.v, d.ph, d.pw, d.dh, d.dw,
                 (d.flags & GBCONV_FLAG_RELU) ? 1 : 0,
                 (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr, fz.alpha, fz.z};
    const size_t smem = (size_t)d.R * d.S * d.C * (d.C / d.G) * 4;
    if (d.in_dtype == GBCONV_F32) return launch_cg<float, float>(d, x, w, y, smem, prm, st);
    if (d.out_dtype == GBCONV_F32)
        return launch_cg<__nv_bfloat16, float>(d, x, w, y, smem, prm, st);
    return launch_cg<__nv_bfloat16, __nv_bfloat16>(d, x, w, y, smem, prm, st);
}

}  // namespace gbc
