// simt.cu -- CUDA-core implicit-GEMM convolution kernels: FP32 FFMA with FP32
// accumulation, no tensor cores, any layout / stride / padding / dilation.
//
// These are the "plain FP32 kernel" of the library (forward of the
// six-nested-loop convolution of the paper's Sec. 1 / Sec. 5.A, reorganised
// as an implicit GEMM the way Sec. 5.B organises it as im2col + GEMM, but
// without materialising the im2col matrix) and the CUDA-core fallback for the
// backward passes (Sec. 5.B) that the tensor-core kernels do not cover.
//
// One CTA computes a 128 x 64 output tile with 256 threads (8 x 4 outputs per
// thread). The reduction runs over k-tiles of 16 elements; every k-tile has a
// fixed filter tap (r, s), so no per-element division is needed. Global loads
// for k-tile t+1 go to registers while k-tile t is multiplied out of shared
// memory (double buffer, one barrier per k-tile).
#include <cuda_bf16.h>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;
constexpr int APAD = 4, BPAD = 4;

template <typename T>
__device__ __forceinline__ float ldf(const T *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
// Coherent load (the residual may be the output tensor itself).
__device__ __forceinline__ float ldz(const float *p) { return *p; }
__device__ __forceinline__ float ldz(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <typename T>
__device__ __forceinline__ void stf(T *p, float v);
template <>
__device__ __forceinline__ void stf<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}

struct DimsK {  // the kernel-side copy of the problem
    int N, C, H, W, K, R, S, P, Q, u, v, ph, pw, dh, dw;
    int Cg, Kg;    // channels per group (forward with groups; else C and K)
};

__host__ DimsK to_k(const Dims &d) {
    return DimsK{d.N, d.C, d.H, d.W, d.K, d.R, d.S, d.P, d.Q, d.u, d.v, d.ph, d.pw, d.dh, d.dw,
                 d.C / d.G, d.K / d.G};
}

// ---------------------------------------------------------------------------
// Shared main loop. The loader L provides:
//   A_KFAST / B_KFAST   which thread->element mapping its loads use
//   begin(t)            per-thread set-up for this CTA's tile
//   kt_begin(), kt_end()
//   load_a(kt, ra[8]), load_b(kt, rb[4])
//   epilogue(acc, tm, tn)
// Mapping of the 8 A elements of thread t: A_KFAST: (k = t%16, m = t/16 + 16i)
// else (m = t%128, k = t/128 + 2i). B elements: B_KFAST: (k = t%16,
// n = t/16 + 16i) else (n = t%64, k = t/64 + 4i).
// ---------------------------------------------------------------------------
template <class L>
__global__ void __launch_bounds__(NT) simt_igemm(L ldr) {
    __shared__ __align__(16) float As[2][BK][BM + APAD];
    __shared__ __align__(16) float Bs[2][BK][BN + BPAD];
    const int t = threadIdx.x;
    const int tm = t % 16, tn = t / 16;
    ptx::griddep_wait();
    ldr.begin(t);
    const int k0 = ldr.kt_begin(), k1 = ldr.kt_end();
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    float ra[8], rb[4];
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int k = L::A_KFAST ? (t % 16) : (t / 128 + 2 * i);
            int m = L::A_KFAST ? (t / 16 + 16 * i) : (t % 128);
            As[buf][k][m] = ra[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int k = L::B_KFAST ? (t % 16) : (t / 64 + 4 * i);
            int n = L::B_KFAST ? (t / 16 + 16 * i) : (t % 64);
            Bs[buf][k][n] = rb[i];
        }
    };
    if (k0 < k1) {
        ldr.load_a(k0, ra);
        ldr.load_b(k0, rb);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int kt = k0; kt < k1; ++kt) {
        const bool more = kt + 1 < k1;
        if (more) {
            ldr.load_a(kt + 1, ra);
            ldr.load_b(kt + 1, rb);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][tm * 8]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][tm * 8 + 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tn * 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if (t == 0) ptx::griddep_launch();
    ldr.epilogue(acc, tm, tn);
}

// ---------------------------------------------------------------------------
// Forward: GEMM rows m = (n,p,q) over N*P*Q, columns = output channel k,
// reduction over (r, s, c) with 16 channels of one tap per k-tile. With
// channel groups, grid layer z = group g: columns are the group's K/G output
// channels and the reduction runs over its C/G input channels.
// ---------------------------------------------------------------------------
template <typename Ti, typename To, bool NHWC>
struct FwdLoader {
    static constexpr bool A_KFAST = NHWC;  // NHWC: channels contiguous
    static constexpr bool B_KFAST = true;
    DimsK d;
    const Ti *x;
    const Ti *w;
    const float *bias;
    To *y;
    int relu;
    int cb;  // channel blocks of 16
    const float *alpha;  // fused: per-channel scale (may be null)
    const To *z;         // fused: residual of y's shape and layout (may be null)
    // per-thread state
    int m0, n0, t;
    int cx0, k0g;  // this group's first input and output channel
    long long xb[8];
    int hb[8], wb[8];

    __device__ void begin(int tid) {
        t = tid;
        m0 = blockIdx.x * BM;
        n0 = blockIdx.y * BN;
        cx0 = blockIdx.z * d.Cg;
        k0g = blockIdx.z * d.Kg;
        const long long M = (long long)d.N * d.P * d.Q;
        const int cnt = NHWC ? 8 : 1;
        for (int i = 0; i < cnt; ++i) {
            long long m = m0 + (NHWC ? (t / 16 + 16 * i) : (t % 128));
            if (m < M) {
                int q = (int)(m % d.Q);
                long long r = m / d.Q;
                int p = (int)(r % d.P);
                int n = (int)(r / d.P);
                xb[i] = (long long)n * d.H * d.W * d.C;
                hb[i] = p * d.u - d.ph;
                wb[i] = q * d.v - d.pw;
            } else {
                xb[i] = 0;
                hb[i] = -(1 << 29);  // never in range
                wb[i] = 0;
            }
        }
    }
    __device__ int kt_begin() const { return 0; }
    __device__ int kt_end() const { return d.R * d.S * cb; }

    __device__ void load_a(int kt, float (&ra)[8]) const {
        const int rs = kt / cb, c0 = (kt - rs * cb) * BK;
        const int r = rs / d.S, s = rs - r * d.S;
        if (NHWC) {
            const int c = c0 + t % 16;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int h = hb[i] + r * d.dh, ww = wb[i] + s * d.dw;
                bool ok = c < d.Cg && h >= 0 && h < d.H && ww >= 0 && ww < d.W;
                ra[i] = ok ? ldf(x + xb[i] + ((long long)h * d.W + ww) * d.C + cx0 + c) : 0.f;
            }
        } else {
            int h = hb[0] + r * d.dh, ww = wb[0] + s * d.dw;
            bool okp = h >= 0 && h < d.H && ww >= 0 && ww < d.W;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int c = c0 + t / 128 + 2 * i;
                bool ok = okp && c < d.Cg;
                ra[i] = ok ? ldf(x + xb[0] + ((long long)(cx0 + c) * d.H + h) * d.W + ww) : 0.f;
            }
        }
    }
    __device__ void load_b(int kt, float (&rb)[4]) const {
        const int rs = kt / cb, c0 = (kt - rs * cb) * BK;
        const int r = rs / d.S, s = rs - r * d.S;
        const int c = c0 + t % 16;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int kl = n0 + t / 16 + 16 * i;  // output channel within the group
            bool ok = c < d.Cg && kl < d.Kg;
            long long k = k0g + kl;
            long long off = NHWC ? ((k * d.R + r) * d.S + s) * d.Cg + c
                                 : ((k * d.Cg + c) * d.R + r) * d.S + s;
            rb[i] = ok ? ldf(w + off) : 0.f;
        }
    }
    __device__ void epilogue(const float (&acc)[8][4], int tm, int tn) const {
        const long long M = (long long)d.N * d.P * d.Q;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            long long m = m0 + tm * 8 + i;
            if (m >= M) continue;
            int q = (int)(m % d.Q);
            long long rr = m / d.Q;
            int p = (int)(rr % d.P);
            int n = (int)(rr / d.P);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int kl = n0 + tn * 4 + j;
                if (kl >= d.Kg) continue;
                const int k = k0g + kl;
                float v = acc[i][j];
                long long off = NHWC ? m * d.K + k : (((long long)n * d.K + k) * d.P + p) * d.Q + q;
                if (alpha) v = v * alpha[k];
                if (bias) v = bias[k] + v;
                if (z) v = v + ldz(z + off);
                if (relu) v = fmaxf(v, 0.f);
                stf(y + off, v);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Data gradient: GEMM rows m = (n,h,w) over N*H*W, columns = input channel c,
// reduction over (r, s, k) with 16 output channels of one tap per k-tile:
//   dx[n,c,h,w] = sum_{k,r,s} g[n,k,p,q] w[k,c,r,s],  p = (h + ph - r*dh)/u
// where the division must be exact and 0 <= p < P (likewise q).
// ---------------------------------------------------------------------------
template <typename Ti, typename To, bool NHWC>
struct DgradLoader {
    static constexpr bool A_KFAST = NHWC;
    static constexpr bool B_KFAST = false;
    DimsK d;
    const Ti *g;
    const Ti *w;
    To *dx;
    int kb;  // output-channel blocks of 16 (of one group)
    int m0, n0, t;
    int cx0, k0g;  // this group's first input and output channel (grid layer z = group)
    long long gb[8];
    int hh[8], wq[8];

    __device__ void begin(int tid) {
        t = tid;
        m0 = blockIdx.x * BM;
        n0 = blockIdx.y * BN;
        cx0 = blockIdx.z * d.Cg;
        k0g = blockIdx.z * d.Kg;
        const long long M = (long long)d.N * d.H * d.W;
        const int cnt = NHWC ? 8 : 1;
        for (int i = 0; i < cnt; ++i) {
            long long m = m0 + (NHWC ? (t / 16 + 16 * i) : (t % 128));
            if (m < M) {
                int ww = (int)(m % d.W);
                long long r = m / d.W;
                int h = (int)(r % d.H);
                int n = (int)(r / d.H);
                gb[i] = (long long)n * d.P * d.Q * d.K;
                hh[i] = h + d.ph;
                wq[i] = ww + d.pw;
            } else {
                gb[i] = 0;
                hh[i] = -(1 << 29);
                wq[i] = -(1 << 29);
            }
        }
    }
    __device__ int kt_begin() const { return 0; }
    __device__ int kt_end() const { return d.R * d.S * kb; }

    __device__ __forceinline__ bool tap(int i, int r, int s, int &p, int &q) const {
        int pn = hh[i] - r * d.dh, qn = wq[i] - s * d.dw;
        if (pn < 0 || qn < 0) return false;
        p = pn / d.u;
        q = qn / d.v;
        return p * d.u == pn && q * d.v == qn && p < d.P && q < d.Q;
    }
    __device__ void load_a(int kt, float (&ra)[8]) const {
        const int rs = kt / kb, k0 = (kt - rs * kb) * BK;
        const int r = rs / d.S, s = rs - r * d.S;
        if (NHWC) {
            const int k = k0 + t % 16;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int p, q;
                bool ok = k < d.Kg && tap(i, r, s, p, q);
                ra[i] = ok ? ldf(g + gb[i] + ((long long)p * d.Q + q) * d.K + k0g + k) : 0.f;
            }
        } else {
            int p = 0, q = 0;
            bool okp = tap(0, r, s, p, q);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int k = k0 + t / 128 + 2 * i;
                bool ok = okp && k < d.Kg;
                ra[i] = ok ? ldf(g + gb[0] + ((long long)(k0g + k) * d.P + p) * d.Q + q) : 0.f;
            }
        }
    }
    __device__ void load_b(int kt, float (&rb)[4]) const {
        const int rs = kt / kb, k0 = (kt - rs * kb) * BK;
        const int r = rs / d.S, s = rs - r * d.S;
        const int c = n0 + t % 64;  // input channel within the group
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int kl = k0 + t / 64 + 4 * i;
            bool ok = c < d.Cg && kl < d.Kg;
            long long k = k0g + kl;
            long long off = NHWC ? ((k * d.R + r) * d.S + s) * d.Cg + c
                                 : ((k * d.Cg + c) * d.R + r) * d.S + s;
            rb[i] = ok ? ldf(w + off) : 0.f;
        }
    }
    __device__ void epilogue(const float (&acc)[8][4], int tm, int tn) const {
        const long long M = (long long)d.N * d.H * d.W;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            long long m = m0 + tm * 8 + i;
            if (m >= M) continue;
            int ww = (int)(m % d.W);
            long long rr = m / d.W;
            int h = (int)(rr % d.H);
            int n = (int)(rr / d.H);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int cl = n0 + tn * 4 + j;
                if (cl >= d.Cg) continue;
                const int c = cx0 + cl;
                long long off = NHWC ? m * d.C + c : (((long long)n * d.C + c) * d.H + h) * d.W + ww;
                stf(dx + off, acc[i][j]);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Weight gradient partial sums. blockIdx.z = filter tap (r, s); blockIdx.y =
// reduction slice. GEMM rows = output channel k, columns = input channel c,
// reduction over output pixels (n, p, q) in runs of 16 along q:
//   part[slice][k,c,r,s] = sum over this slice's pixels of g[n,k,p,q] x[n,c,h,w]
// ---------------------------------------------------------------------------
template <typename Ti, bool NHWC>
struct WgradLoader {
    static constexpr bool A_KFAST = !NHWC;  // NHWC g: k contiguous (rows)
    static constexpr bool B_KFAST = !NHWC;  // NHWC x: c contiguous (columns)
    DimsK d;
    const Ti *x;
    const Ti *g;
    float *part;
    int slices, qb, m_tiles;
    int m0, n0, t, r, s, kt0, kt1;
    int cx0, k0g;  // this group's first input and output channel

    __device__ void begin(int tid) {
        t = tid;
        m0 = (blockIdx.x % m_tiles) * BM;
        n0 = (blockIdx.x / m_tiles) * BN;
        const int RS = d.R * d.S;
        const int grp = blockIdx.z / RS, tap = blockIdx.z - grp * RS;  // grid layer z = (group, tap)
        cx0 = grp * d.Cg;
        k0g = grp * d.Kg;
        r = tap / d.S;
        s = tap - r * d.S;
        long long total = (long long)d.N * d.P * qb;
        kt0 = (int)(total * blockIdx.y / slices);
        kt1 = (int)(total * (blockIdx.y + 1) / slices);
    }
    __device__ int kt_begin() const { return kt0; }
    __device__ int kt_end() const { return kt1; }

    // k-tile -> image row (n, p) and first column q0
    __device__ __forceinline__ void row(int kt, int &n, int &p, int &q0) const {
        int rowi = kt / qb;
        q0 = (kt - rowi * qb) * BK;
        p = rowi % d.P;
        n = rowi / d.P;
    }
    __device__ void load_a(int kt, float (&ra)[8]) const {
        int n, p, q0;
        row(kt, n, p, q0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int kl = A_KFAST ? (t % 16) : (t / 128 + 2 * i);
            int ml = A_KFAST ? (t / 16 + 16 * i) : (t % 128);
            int q = q0 + kl, kl2 = m0 + ml;
            bool ok = q < d.Q && kl2 < d.Kg;
            const long long k = k0g + kl2;
            long long off = NHWC ? (((long long)n * d.P + p) * d.Q + q) * d.K + k
                                 : (((long long)n * d.K + k) * d.P + p) * d.Q + q;
            ra[i] = ok ? ldf(g + off) : 0.f;
        }
    }
    __device__ void load_b(int kt, float (&rb)[4]) const {
        int n, p, q0;
        row(kt, n, p, q0);
        const int h = p * d.u + r * d.dh - d.ph;
        const bool okh = h >= 0 && h < d.H;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int kl = B_KFAST ? (t % 16) : (t / 64 + 4 * i);
            int nl = B_KFAST ? (t / 16 + 16 * i) : (t % 64);
            int q = q0 + kl, cl = n0 + nl;
            int ww = q * d.v + s * d.dw - d.pw;
            bool ok = okh && q < d.Q && cl < d.Cg && ww >= 0 && ww < d.W;
            const long long c = cx0 + cl;
            long long off = NHWC ? (((long long)n * d.H + h) * d.W + ww) * d.C + c
                                 : (((long long)n * d.C + c) * d.H + h) * d.W + ww;
            rb[i] = ok ? ldf(x + off) : 0.f;
        }
    }
    __device__ void epilogue(const float (&acc)[8][4], int tm, int tn) const {
        float *out = part + (long long)blockIdx.y * d.K * d.Cg * d.R * d.S;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int kl = m0 + tm * 8 + i;
            if (kl >= d.Kg) continue;
            const long long k = k0g + kl;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int c = n0 + tn * 4 + j;  // within the group (the filter holds C/G channels)
                if (c >= d.Cg) continue;
                long long off = NHWC ? ((k * d.R + r) * d.S + s) * d.Cg + c
                                     : ((k * d.Cg + c) * d.R + r) * d.S + s;
                out[off] = acc[i][j];
            }
        }
    }
};

template <class L>
gbconv_status_t launch(const L &ldr, dim3 grid, cudaStream_t st) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return GBCONV_OK;
    return cuda_status(launch_pdl(simt_igemm<L>, grid, dim3(NT), 0, st, ldr));
}

template <typename Ti, typename To>
gbconv_status_t fwd_typed(const Dims &d, const void *x, const void *w, const float *bias, void *y,
                          cudaStream_t st, const Fused &fz) {
    long long M = d.M();
    const int Kg = d.K / d.G, Cg = d.C / d.G;
    if (d.G > 65535) return GBCONV_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Kg + BN - 1) / BN), (unsigned)d.G);
    int relu = (d.flags & GBCONV_FLAG_RELU) ? 1 : 0;
    const float *b = (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr;
    int cb = (Cg + BK - 1) / BK;
    if (d.layout == GBCONV_NHWC) {
        FwdLoader<Ti, To, true> L{to_k(d), (const Ti *)x, (const Ti *)w, b, (To *)y, relu, cb,
                                  fz.alpha, (const To *)fz.z};
        return launch(L, grid, st);
    }
    FwdLoader<Ti, To, false> L{to_k(d), (const Ti *)x, (const Ti *)w, b, (To *)y, relu, cb,
                               fz.alpha, (const To *)fz.z};
    return launch(L, grid, st);
}

template <typename Ti, typename To>
gbconv_status_t dgrad_typed(const Dims &d, const void *g, const void *w, void *dx,
                            cudaStream_t st) {
    long long M = (long long)d.N * d.H * d.W;
    const int Cg = d.C / d.G, Kg = d.K / d.G;
    if (d.G > 65535) return GBCONV_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Cg + BN - 1) / BN), (unsigned)d.G);
    int kb = (Kg + BK - 1) / BK;
    if (d.layout == GBCONV_NHWC) {
        DgradLoader<Ti, To, true> L{to_k(d), (const Ti *)g, (const Ti *)w, (To *)dx, kb};
        return launch(L, grid, st);
    }
    DgradLoader<Ti, To, false> L{to_k(d), (const Ti *)g, (const Ti *)w, (To *)dx, kb};
    return launch(L, grid, st);
}

template <typename Ti>
gbconv_status_t wgrad_typed(const Dims &d, const void *x, const void *g, float *ws, int slices,
                            cudaStream_t st) {
    const int Cg = d.C / d.G, Kg = d.K / d.G;
    int m_tiles = (Kg + BM - 1) / BM, n_tiles = (Cg + BN - 1) / BN;
    int qb = (d.Q + BK - 1) / BK;
    if ((long long)d.R * d.S * d.G > 65535) return GBCONV_ERR_UNSUPPORTED;
    dim3 grid((unsigned)(m_tiles * n_tiles), (unsigned)slices, (unsigned)(d.R * d.S * d.G));
    if (d.layout == GBCONV_NHWC) {
        WgradLoader<Ti, true> L{to_k(d), (const Ti *)x, (const Ti *)g, ws, slices, qb, m_tiles};
        return launch(L, grid, st);
    }
    WgradLoader<Ti, false> L{to_k(d), (const Ti *)x, (const Ti *)g, ws, slices, qb, m_tiles};
    return launch(L, grid, st);
}

}  // namespace

gbconv_status_t launch_simt_fwd(const Dims &d, const void *x, const void *w, const float *bias,
                                void *y, cudaStream_t st, const Fused &fz) {
    if (d.in_dtype == GBCONV_F32 && d.out_dtype == GBCONV_F32)
        return fwd_typed<float, float>(d, x, w, bias, y, st, fz);
    if (d.in_dtype == GBCONV_BF16 && d.out_dtype == GBCONV_F32)
        return fwd_typed<__nv_bfloat16, float>(d, x, w, bias, y, st, fz);
    if (d.in_dtype == GBCONV_BF16 && d.out_dtype == GBCONV_BF16)
        return fwd_typed<__nv_bfloat16, __nv_bfloat16>(d, x, w, bias, y, st, fz);
    return GBCONV_ERR_UNSUPPORTED;
}

gbconv_status_t launch_simt_dgrad(const Dims &d, const void *g, const void *w, void *dx,
                                  cudaStream_t st) {
    if (d.in_dtype == GBCONV_F32 && d.out_dtype == GBCONV_F32)
        return dgrad_typed<float, float>(d, g, w, dx, st);
    if (d.in_dtype == GBCONV_BF16 && d.out_dtype == GBCONV_F32)
        return dgrad_typed<__nv_bfloat16, float>(d, g, w, dx, st);
    if (d.in_dtype == GBCONV_BF16 && d.out_dtype == GBCONV_BF16)
        return dgrad_typed<__nv_bfloat16, __nv_bfloat16>(d, g, w, dx, st);
    return GBCONV_ERR_UNSUPPORTED;
}

gbconv_status_t launch_simt_wgrad_partials(const Dims &d, const void *x, const void *g,
                                           float *ws, int slices, cudaStream_t st) {
    if (d.in_dtype == GBCONV_F32) return wgrad_typed<float>(d, x, g, ws, slices, st);
    if (d.in_dtype == GBCONV_BF16) return wgrad_typed<__nv_bfloat16>(d, x, g, ws, slices, st);
    return GBCONV_ERR_UNSUPPORTED;
}

}  // namespace gbc
