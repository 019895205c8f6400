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
//
// Two kernels share that arithmetic:
//  - the staged kernel (BF16 input): a persistent block takes bands of TR
//    output rows of one image; the band's input rows, each a contiguous W*C
//    run in NHWC, arrive in shared memory by bulk asynchronous copies (one per
//    row, completing on an mbarrier), two bands in flight, between zeroed
//    padding columns, so the arithmetic reads shared memory only;
//  - the direct kernel (FP32 input, or a band that does not fit): every
//    thread reads its taps from global memory.
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
// Staged kernel: filter + two band stages + two mbarriers. Bands that fit in
// DWT_SMEM_PAIR run two blocks per SM, otherwise one up to DWT_SMEM_MAX.
constexpr int DWT_SMEM_PAIR = 110 * 1024;
constexpr int DWT_SMEM_MAX = 200 * 1024;
constexpr int DWT_MAX_TR = 16;

struct DwParams {
    int N, C, H, W, P, Q, R, S, u, v, ph, pw, dh, dw;
    int relu;
    const float *bias, *alpha;
    const void *z;
    // staged kernel: output rows per band, input rows per band, padded row
    // width (columns), bands per image, bands
    int TR, HB, WP, bands_per_image, nbands;
    Guard guard;
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
// filter row's loads are issued before the first multiply. Global rows are
// read through a pointer, staged rows by 32-bit shared-memory address.
__device__ __forceinline__ uint4 ldraw(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint4 *>(p);
}
__device__ __forceinline__ uint4 ldraw_s(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}
// BF16 is the upper half of an FP32 word, so widening is exact bit
// placement: the low element of a 32-bit pair shifted up, the high one masked.
__device__ __forceinline__ void unpack8(const uint4 &u, float (&v)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(w[i] << 16);
        v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
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

// (d0, d1) = (a0*b0 + d0, a1*b1 + d1), each rounded once: the packed FP32
// FMA, two lanes' worth of fmaf in one instruction.
__device__ __forceinline__ void ffma2(float &d0, float &d1, float a0, float a1, float b0,
                                      float b1) {
    asm("{\n\t.reg .b64 d, a, b;\n\t"
        "mov.b64 a, {%2, %3};\n\t"
        "mov.b64 b, {%4, %5};\n\t"
        "mov.b64 d, {%0, %1};\n\t"
        "fma.rn.f32x2 d, a, b, d;\n\t"
        "mov.b64 {%0, %1}, d;\n}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// acc[j] += sum_c xv[gb(j) + c] * wv[j*CG + c]: the thread's 8 output
// channels against the CG input channels of each one's group (one channel:
// neighbouring channels pair up in packed FMAs).
template <int CG>
__device__ __forceinline__ void fma8(const float (&xv)[8], const float (&wv)[8 * CG],
                                     float (&acc)[8]) {
    if constexpr (CG == 1) {
#pragma unroll
        for (int j = 0; j < 8; j += 2)
            ffma2(acc[j], acc[j + 1], xv[j], xv[j + 1], wv[j], wv[j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gb = (j / CG) * CG;  // first channel of j's group in the vector
#pragma unroll
            for (int c = 0; c < CG; ++c) acc[j] = fmaf(xv[gb + c], wv[j * CG + c], acc[j]);
        }
    }
}

// Stages the filter [K][R][S][CG] as FP32 in the slot-major layout.
template <typename Ti, int CG>
__device__ __forceinline__ void stage_filter(const Ti *w, float *wsm, int RS, int C) {
    const int cv = C / 8;
    for (int i = threadIdx.x; i < RS * C * CG; i += blockDim.x) {
        const int e = i & 3;
        int t = i >> 2;
        const int cvi = t % cv;
        t /= cv;
        const int f = (t % (2 * CG)) * 4 + e, rs = t / (2 * CG);
        const int k = cvi * 8 + f / CG, c = f % CG;
        wsm[i] = static_cast<float>(w[((long long)k * RS + rs) * CG + c]);
    }
}

// Accumulates filter row r into the thread's PX pixels x 8 channels. xrow
// (global rows) points at channel c0 of the row's column 0, xs (staged rows)
// is its shared-memory address; pixel q0 + a, tap s reads column
// (q0 + a)*v + s*dw - off. CHECK (global rows): columns outside [0, W) and
// pixels at or past Q read zeros. Without CHECK the row is staged in shared
// memory between zero padding columns (off = 0) wide enough for every pixel
// of the last pixel block. SC > 0 (BF16 input only): the filter
// width is the constant SC, so the row's loads are unrolled and issued
// together. UNIT (horizontal stride and dilation 1): the PX pixels' SC taps
// cover only PX + SC - 1 columns, each loaded (and, up to two channels per
// group, converted to FP32) once.
template <typename Ti, int CG, int SC, bool UNIT, int PX, bool CHECK>
__device__ __forceinline__ void row_fma(const Ti *xrow, uint32_t xs, int q0, const DwParams &prm,
                                        int off, const float4 *wt, int cv, float (&acc)[PX][8]) {
    const int C = prm.C;
    auto ld = [&](int col) {  // a BF16 channel vector of column col
        if constexpr (CHECK) {
            return ldraw(reinterpret_cast<const __nv_bfloat16 *>(xrow) + col * C);
        } else {
            return ldraw_s(xs + (uint32_t)(col * C * 2));
        }
    };
    if constexpr (SC > 0 && UNIT) {
        constexpr int NX = PX + SC - 1;
        uint4 xr[NX];
#pragma unroll
        for (int e = 0; e < NX; ++e) {
            const int ww = q0 + e - off;
            xr[e] = (!CHECK || (ww >= 0 && ww < prm.W)) ? ld(ww) : make_uint4(0, 0, 0, 0);
        }
        if constexpr (CG <= 2) {
            float xv[NX][8];
#pragma unroll
            for (int e = 0; e < NX; ++e) unpack8(xr[e], xv[e]);
#pragma unroll
            for (int s = 0; s < SC; ++s) {
                float wv[8 * CG];
                load_taps<CG>(wt + s * 2 * CG * cv, cv, wv);
#pragma unroll
                for (int a = 0; a < PX; ++a) fma8<CG>(xv[a + s], wv, acc[a]);
            }
        } else {
#pragma unroll
            for (int s = 0; s < SC; ++s) {
                float wv[8 * CG];
                load_taps<CG>(wt + s * 2 * CG * cv, cv, wv);
#pragma unroll
                for (int a = 0; a < PX; ++a) {
                    float xv[8];
                    unpack8(xr[a + s], xv);
                    fma8<CG>(xv, wv, acc[a]);
                }
            }
        }
    } else if constexpr (SC > 0) {
        uint4 xr[SC][PX];
#pragma unroll
        for (int s = 0; s < SC; ++s)
#pragma unroll
            for (int a = 0; a < PX; ++a) {
                const int ww = (q0 + a) * prm.v + s * prm.dw - off;
                xr[s][a] = (!CHECK || (q0 + a < prm.Q && ww >= 0 && ww < prm.W))
                               ? ld(ww)
                               : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
        for (int s = 0; s < SC; ++s) {
            float wv[8 * CG];
            load_taps<CG>(wt + s * 2 * CG * cv, cv, wv);
#pragma unroll
            for (int a = 0; a < PX; ++a) {
                float xv[8];
                unpack8(xr[s][a], xv);
                fma8<CG>(xv, wv, acc[a]);
            }
        }
    } else {
        for (int s = 0; s < prm.S; ++s) {
            // this tap's PX input vectors first (all loads in flight), then the math
            float xv[PX][8];
#pragma unroll
            for (int a = 0; a < PX; ++a) {
                const int ww = (q0 + a) * prm.v + s * prm.dw - off;
                if (!CHECK || (q0 + a < prm.Q && ww >= 0 && ww < prm.W)) {
                    if constexpr (CHECK) {
                        load8(xrow + (long long)ww * C, xv[a]);
                    } else {
                        unpack8(ld(ww), xv[a]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) xv[a][j] = 0.f;
                }
            }
            float wv[8 * CG];  // this tap's weights of the thread's 8 output channels
            load_taps<CG>(wt + s * 2 * CG * cv, cv, wv);
#pragma unroll
            for (int a = 0; a < PX; ++a) fma8<CG>(xv[a], wv, acc[a]);
        }
    }
}

// y = act(alpha*acc + b + z) for the thread's pixels of output row p.
template <typename To, int PX>
__device__ __forceinline__ void store_pixels(To *y, const DwParams &prm, int n, int p, int q0,
                                             int c0, float (&acc)[PX][8]) {
    const To *z = static_cast<const To *>(prm.z);
    float al[8], bi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        al[j] = prm.alpha ? prm.alpha[c0 + j] : 1.f;
        bi[j] = prm.bias ? prm.bias[c0 + j] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < PX; ++a) {
        if (q0 + a >= prm.Q) break;
        const long long off = (((long long)n * prm.P + p) * prm.Q + q0 + a) * prm.C + c0;
        float zv[8];
        if (z) load8(z + off, zv);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v = acc[a][j];
            if (prm.alpha) v = v * al[j];
            if (prm.bias) v = bi[j] + v;
            if (z) v = v + zv[j];
            if (prm.relu) v = fmaxf(v, 0.f);
            acc[a][j] = v;
        }
        store8(y + off, acc[a]);
    }
}

// Direct kernel. Work items (PX pixels x 8 channels) are numbered in 32 bits
// (fewer than 2^31, checked on the host).
template <typename Ti, typename To, int CG, int SC, bool UNIT>
__global__ void __launch_bounds__(DW_THREADS, Px<CG>::min_blocks) depthwise_kernel(
    const Ti *__restrict__ x, const Ti *__restrict__ w, To *y, const DwParams prm) {
    constexpr int PX = Px<CG>::v;
    extern __shared__ float4 wsm4[];  // [R*S][2*CG][C/8]
    const int RS = prm.R * prm.S, C = prm.C;  // C = K
    const int cv = C / 8;                     // channel vectors per pixel
    // The filter is a kernel input like x: read it after the dependency wait.
    ptx::griddep_wait();
    stage_filter<Ti, CG>(w, reinterpret_cast<float *>(wsm4), RS, C);
    __syncthreads();
    if (threadIdx.x == 0) ptx::griddep_launch();
    const unsigned qb = (prm.Q + PX - 1) / PX;  // pixel blocks per output row
    const unsigned total = (unsigned)prm.N * prm.P * qb * cv;
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
            row_fma<Ti, CG, SC, UNIT, PX, true>(xrow, 0, q0, prm, prm.pw,
                                                wsm4 + r * prm.S * 2 * CG * cv + c0 / 8, cv, acc);
        }
        store_pixels<To, PX>(y, prm, n, p, q0, c0, acc);
    }
}

// 1-D bulk copy global -> shared completing on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(ptx::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(ptx::smem_addr(bar))
        : "memory");
}

// Staged kernel (BF16 input). Shared memory: filter [R*S][2*CG][C/8] float4,
// two stages [HB][WP][C] BF16 (input columns at pw .. pw+W-1, zeros around),
// two mbarriers. Band b covers output rows p0 .. p0+TR-1 of image n (b =
// n * bands_per_image + p0 / TR) and input rows h0 .. h0+HB-1, h0 = p0*u - ph;
// only rows inside [0, H) are copied and read.
template <typename To, int CG, int SC, bool UNIT>
__global__ void __launch_bounds__(DW_THREADS, 2) depthwise_staged_kernel(
    const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ w, To *y,
    const DwParams prm) {
    constexpr int PX = Px<CG>::v;
    extern __shared__ float4 sm4[];
    const int RS = prm.R * prm.S, C = prm.C, cv = C / 8;
    const float4 *wsm4 = sm4;
    __nv_bfloat16 *stage0 = reinterpret_cast<__nv_bfloat16 *>(sm4 + RS * 2 * CG * cv);
    const int stage_elems = prm.HB * prm.WP * C;  // a multiple of 8
    uint64_t *bar = reinterpret_cast<uint64_t *>(stage0 + 2 * stage_elems);
    const int tid = threadIdx.x;
    if (tid == 0) {
        ptx::mbar_init(&bar[0], 1);
        ptx::mbar_init(&bar[1], 1);
        ptx::fence_mbar_init();
    }
    {  // zero padding columns of both stages (the copies never write them)
        const int padL = prm.pw, padR = prm.WP - prm.pw - prm.W;
        const int pv = (padL + padR) * cv;  // 16-byte vectors per row
        uint4 *s4 = reinterpret_cast<uint4 *>(stage0);
        for (int i = tid; i < 2 * prm.HB * pv; i += blockDim.x) {
            const int e = i % pv, row = i / pv;
            const int col = e / cv, cvi = e % cv;
            const int cc = col < padL ? col : prm.pw + prm.W + (col - padL);
            s4[(row * prm.WP + cc) * cv + cvi] = make_uint4(0, 0, 0, 0);
        }
    }
    const bool skip = prm.guard.skip_loads != 0;
    const uint32_t row_bytes = (uint32_t)prm.W * C * 2;
    // thread 0: the copies of band b into stage st (an arrival without bytes
    // if none of its rows exists; nothing at all under the skip-loads test
    // control, so that the waits run out)
    auto issue = [&](int b, int st) {
        if (skip) return;
        const int n = b / prm.bands_per_image, p0 = (b % prm.bands_per_image) * prm.TR;
        const int h0 = p0 * prm.u - prm.ph;
        const int lo = max(0, -h0), hi = min(prm.HB, prm.H - h0);
        if (hi <= lo) {
            ptx::mbar_arrive(&bar[st]);
            return;
        }
        ptx::mbar_arrive_expect_tx(&bar[st], (uint32_t)(hi - lo) * row_bytes);
        __nv_bfloat16 *dst = stage0 + st * stage_elems + prm.pw * C;
        const __nv_bfloat16 *src = x + ((long long)n * prm.H + h0) * prm.W * C;
        for (int hr = lo; hr < hi; ++hr)
            bulk_load(dst + hr * prm.WP * C, src + (long long)hr * prm.W * C, row_bytes, &bar[st]);
    };
    ptx::griddep_wait();
    if (tid == 0) {
        if ((int)blockIdx.x < prm.nbands) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < prm.nbands) issue(blockIdx.x + gridDim.x, 1);
    }
    stage_filter<__nv_bfloat16, CG>(w, reinterpret_cast<float *>(sm4), RS, C);
    __syncthreads();
    if (tid == 0) ptx::griddep_launch();

    const unsigned qb = (prm.Q + PX - 1) / PX;
    const unsigned items = (unsigned)prm.TR * qb * cv;
    const uint64_t lim = prm.guard.wait_ns;
    volatile int zero = 0;
    int it = 0;
    for (int b = blockIdx.x; b < prm.nbands; b += gridDim.x, ++it) {
        const int st = it & 1;
        const uint32_t par = (it >> 1) & 1;
        // one thread polls; the others sleep in the block barrier, then
        // observe the completed phase themselves (a single test each)
        bool got = true;
        if (tid == 0) got = ptx::mbar_wait(&bar[st], par, lim, &zero);
        if (__syncthreads_or(!got)) {
            // a copy did not complete in time: record it, wait (bounded) for
            // the copies this block still has in flight, and stop
            if (tid == 0) {
                atomicOr(prm.guard.err, DEVERR_TIMEOUT);
                if (!skip) {
                    ptx::mbar_wait(&bar[st], par, lim, &zero);
                    if (b + (int)gridDim.x < prm.nbands)
                        ptx::mbar_wait(&bar[st ^ 1], ((it + 1) >> 1) & 1, lim, &zero);
                }
            }
            return;
        }
        if (tid != 0) ptx::mbar_try_wait(&bar[st], par);
        const int n = b / prm.bands_per_image, p0 = (b % prm.bands_per_image) * prm.TR;
        const int h0 = p0 * prm.u - prm.ph;
        const uint32_t sx = ptx::smem_addr(stage0 + st * stage_elems);
        for (unsigned i = tid; i < items; i += blockDim.x) {
            const int c0 = (int)(i % (unsigned)cv) * 8;
            const unsigned t = i / (unsigned)cv;
            const int q0 = (int)(t % qb) * PX;
            const int pr = (int)(t / qb);
            const int p = p0 + pr;
            if (p >= prm.P) continue;  // ragged last band of an image
            float acc[PX][8];
#pragma unroll
            for (int a = 0; a < PX; ++a)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[a][j] = 0.f;
            for (int r = 0; r < prm.R; ++r) {
                const int hr = pr * prm.u + r * prm.dh;
                if (h0 + hr < 0 || h0 + hr >= prm.H) continue;
                row_fma<__nv_bfloat16, CG, SC, UNIT, PX, false>(
                    nullptr, sx + (uint32_t)((hr * prm.WP * C + c0) * 2), q0, prm, 0,
                    wsm4 + r * prm.S * 2 * CG * cv + c0 / 8, cv, acc);
            }
            store_pixels<To, PX>(y, prm, n, p, q0, c0, acc);
        }
        __syncthreads();  // stage st fully read before it is refilled
        if (tid == 0 && b + 2 * (int)gridDim.x < prm.nbands) issue(b + 2 * gridDim.x, st);
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
    return cuda_status(launch_pdl(depthwise_kernel<Ti, To, CG, SC, UNIT>, dim3(grid), dim3(DW_THREADS),
                                  smem, st, static_cast<const Ti *>(x), static_cast<const Ti *>(w),
                                  static_cast<To *>(y), prm));
}

template <typename To, int CG, int SC, bool UNIT = false>
gbconv_status_t launch_staged(const void *x, const void *w, void *y, size_t smem,
                              const DwParams &prm, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(depthwise_staged_kernel<To, CG, SC, UNIT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, DWT_SMEM_MAX);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    const int per_sm = smem <= (size_t)DWT_SMEM_PAIR ? 2 : 1;
    const unsigned grid = (unsigned)std::min(prm.nbands, sm_count() * per_sm);
    return cuda_status(launch_pdl(depthwise_staged_kernel<To, CG, SC, UNIT>, dim3(grid),
                                  dim3(DW_THREADS), smem, st,
                                  static_cast<const __nv_bfloat16 *>(x),
                                  static_cast<const __nv_bfloat16 *>(w), static_cast<To *>(y), prm));
}

// Band plan of the staged kernel: the most output rows per band whose two
// stages fit two blocks per SM, else one block per SM; false if not even a
// one-row band fits. Returns the dynamic shared memory size in smem.
bool staged_plan(const Dims &d, DwParams &prm, size_t &smem) {
    const int cg = d.C / d.G, px = cg == 8 ? 2 : 4;
    const int qb = (d.Q + px - 1) / px;
    const int WP = std::max(d.pw + d.W, (qb * px - 1) * d.v + (d.S - 1) * d.dw + 1);
    const long long wbytes = (long long)d.R * d.S * d.C * cg * 4;
    const long long row = (long long)WP * d.C * 2;
    for (const long long cap : {(long long)DWT_SMEM_PAIR, (long long)DWT_SMEM_MAX}) {
        for (int tr = std::min(d.P, DWT_MAX_TR); tr >= 1; --tr) {
            const int hb = (tr - 1) * d.u + (d.R - 1) * d.dh + 1;
            const long long bytes = wbytes + 2 * hb * row + 16;
            if (bytes > cap) continue;
            prm.TR = tr;
            prm.HB = hb;
            prm.WP = WP;
            prm.bands_per_image = (d.P + tr - 1) / tr;
            prm.nbands = d.N * prm.bands_per_image;
            smem = (size_t)bytes;
            return true;
        }
    }
    return false;
}

template <typename To>
gbconv_status_t launch_staged_cg(const Dims &d, const void *x, const void *w, void *y,
                                 size_t smem, const DwParams &prm, cudaStream_t st) {
    const bool unit = d.v == 1 && d.dw == 1;
    if (d.S == 3 && d.C == d.G)
        return unit ? launch_staged<To, 1, 3, true>(x, w, y, smem, prm, st)
                    : launch_staged<To, 1, 3>(x, w, y, smem, prm, st);
    if (d.S == 3 && d.C == 2 * d.G)
        return unit ? launch_staged<To, 2, 3, true>(x, w, y, smem, prm, st)
                    : launch_staged<To, 2, 3>(x, w, y, smem, prm, st);
    if constexpr (std::is_same<To, __nv_bfloat16>::value) {
        if (d.S == 3 && d.C == 4 * d.G)
            return unit ? launch_staged<To, 4, 3, true>(x, w, y, smem, prm, st)
                        : launch_staged<To, 4, 3>(x, w, y, smem, prm, st);
    }
    switch (d.C / d.G) {
        case 1: return launch_staged<To, 1, 0>(x, w, y, smem, prm, st);
        case 2: return launch_staged<To, 2, 0>(x, w, y, smem, prm, st);
        case 4: return launch_staged<To, 4, 0>(x, w, y, smem, prm, st);
        default: return launch_staged<To, 8, 0>(x, w, y, smem, prm, st);
    }
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
                 (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr, fz.alpha, fz.z,
                 0, 0, 0, 0, 0, Guard{}};
    if (d.in_dtype == GBCONV_BF16) {
        size_t smem = 0;
        if (staged_plan(d, prm, smem)) {
            prm.guard = make_guard();
            if (!prm.guard.err) return GBCONV_ERR_CUDA;
            if (d.out_dtype == GBCONV_F32) return launch_staged_cg<float>(d, x, w, y, smem, prm, st);
            return launch_staged_cg<__nv_bfloat16>(d, x, w, y, smem, prm, st);
        }
    }
    const size_t smem = (size_t)d.R * d.S * d.C * (d.C / d.G) * 4;
    if (d.in_dtype == GBCONV_F32) return launch_cg<float, float>(d, x, w, y, smem, prm, st);
    if (d.out_dtype == GBCONV_F32)
        return launch_cg<__nv_bfloat16, float>(d, x, w, y, smem, prm, st);
    return launch_cg<__nv_bfloat16, __nv_bfloat16>(d, x, w, y, smem, prm, st);
}

}  // namespace gbc
