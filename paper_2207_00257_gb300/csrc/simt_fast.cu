// simt_fast.cu -- the plain FP32 forward convolution for NHWC tensors whose
// channel counts are multiples of 4: FP32 FFMA on the CUDA cores, FP32
// accumulation, no tensor cores (the six-nested-loop convolution of the
// paper's Sec. 1 / Sec. 5.A, organised as the implicit GEMM of Sec. 5.B
// without materialising the im2col matrix).
//
// GEMM: rows m = (n, p, q) over N*P*Q, columns = output channel k, reduction
// over (r, s, c) in k-tiles of 16 channels of one filter tap.
//  * CTA tile 128 x BN (BN = 128 or 64), 256 threads, 8 x (BN/16) outputs per
//    thread, held as two 4-row halves 64 rows apart (and, for BN = 128, two
//    4-column halves 64 columns apart), so that the shared-memory fragment
//    reads of a warp are conflict-free 16-byte loads.
//  * Global loads are 16-byte vectors (4 consecutive channels of one pixel,
//    or of one filter row); the next k-tile's vectors are loaded into
//    registers while the current one is multiplied out of shared memory
//    (double buffer, one barrier per k-tile).
//  * Per k-tile and thread: 8 x BN/16 x 16 FFMAs against 16 x (2 + BN/64)
//    16-byte shared loads.
// Epilogue: optional per-channel scale, bias, residual, ReLU, 16-byte stores.
#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int FM = 128, FK = 16, FT = 256;  // FT: threads of the 128-wide tile
constexpr int FPAD = 4;  // row padding of the shared tiles (floats)

struct FastArgs {
    int N, C, H, W, K, P, Q, S, RS, u, v, ph, pw, dh, dw;
    int cb;      // channel blocks of 16 per tap
    int ktiles;  // R * S * cb
    int M;  // all offsets fit 31 bits (checked on the host)
    const float *x, *w, *bias, *alpha;
    const float *z;  // residual of y's shape (may be y itself) or null
    float *y;
    int relu;
};

// NT threads: 16 row groups x NT/16 column groups, 8 x TN outputs each
// (TN = 16*BN/NT). Per k-step a thread reads 2 + TN/4 16-byte fragments for
// 8*TN FFMAs: the 8 x 8 forms (128 x 128 on 256 threads, 128 x 64 on 128
// threads) balance shared-memory wavefronts against FFMA issue, the 8 x 4
// form (128 x 64 on 256 threads) is bound by shared memory. Blocks per SM:
// 4 for 128 threads, 3 for 128 x 64 on 256, 2 for 128 x 128 (registers).
template <int BN, int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 4 : (BN == 64 ? 3 : 2))
    simt_fast_fwd(const FastArgs a) {
    constexpr int TN = 16 * BN / NT;       // columns per thread (8 or 4)
    constexpr int RP = NT / 4;             // rows loaded per pass
    constexpr int AP = FM / RP;            // pixel vectors per thread per k-tile
    constexpr int BV = BN / RP;            // filter vectors per thread per k-tile
    __shared__ __align__(16) float As[2][FK][FM + FPAD];
    __shared__ __align__(16) float Bs[2][FK][BN + FPAD];
    const int t = threadIdx.x;
    const int tm = t & 15, tn = t >> 4;
    const int m0 = blockIdx.x * FM;
    const int n0 = blockIdx.y * BN;
    ptx::griddep_wait();

    // this thread's AP pixels (A vectors) and BV filter rows (B vectors)
    const int cq = (t & 3) * 4;  // channel quad inside the k-tile
    int xbase[AP];
    int hb[AP], wb[AP];
#pragma unroll
    for (int i = 0; i < AP; ++i) {
        const int m = m0 + (t >> 2) + RP * i;
        if (m < a.M) {
            const int q = m % a.Q;
            const int r = m / a.Q;
            const int p = r % a.P;
            const int n = r / a.P;
            xbase[i] = n * a.H * a.W * a.C;
            hb[i] = p * a.u - a.ph;
            wb[i] = q * a.v - a.pw;
        } else {
            xbase[i] = 0;
            hb[i] = -(1 << 29);
            wb[i] = 0;
        }
    }
    int krow[BV];
#pragma unroll
    for (int i = 0; i < BV; ++i) krow[i] = n0 + (t >> 2) + RP * i;

    float4 ra[AP], rb[BV];
    auto load = [&](int kt) {
        const int rs = kt / a.cb, c = (kt - rs * a.cb) * FK + cq;
        const int r = rs / a.S, s = rs - r * a.S;
#pragma unroll
        for (int i = 0; i < AP; ++i) {
            const int h = hb[i] + r * a.dh, ww = wb[i] + s * a.dw;
            const bool ok = c < a.C && h >= 0 && h < a.H && ww >= 0 && ww < a.W;
            ra[i] = ok ? __ldg(reinterpret_cast<const float4 *>(
                             a.x + xbase[i] + (h * a.W + ww) * a.C + c))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < BV; ++i) {
            const bool ok = c < a.C && krow[i] < a.K;
            rb[i] = ok ? __ldg(reinterpret_cast<const float4 *>(a.w + (krow[i] * a.RS + rs) * a.C + c))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
        const int mr = t >> 2;
#pragma unroll
        for (int i = 0; i < AP; ++i) {
            As[buf][cq + 0][mr + RP * i] = ra[i].x;
            As[buf][cq + 1][mr + RP * i] = ra[i].y;
            As[buf][cq + 2][mr + RP * i] = ra[i].z;
            As[buf][cq + 3][mr + RP * i] = ra[i].w;
        }
#pragma unroll
        for (int i = 0; i < BV; ++i) {
            Bs[buf][cq + 0][mr + RP * i] = rb[i].x;
            Bs[buf][cq + 1][mr + RP * i] = rb[i].y;
            Bs[buf][cq + 2][mr + RP * i] = rb[i].z;
            Bs[buf][cq + 3][mr + RP * i] = rb[i].w;
        }
    };

    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    if (a.ktiles > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int kt = 0; kt < a.ktiles; ++kt) {
        const bool more = kt + 1 < a.ktiles;
        if (more) load(kt + 1);
#pragma unroll
        for (int k = 0; k < FK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][tm * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + tm * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float bv[TN];
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tn * 4]);
            bv[0] = b0.x;
            bv[1] = b0.y;
            bv[2] = b0.z;
            bv[3] = b0.w;
            if constexpr (TN == 8) {
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][BN / 2 + tn * 4]);
                bv[4] = b1.x;
                bv[5] = b1.y;
                bv[6] = b1.z;
                bv[7] = b1.w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if (t == 0) ptx::griddep_launch();

    // epilogue: rows tm*4 + i (+64), columns tn*4 + j (+BN/2)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? tm * 4 + i : 64 + tm * 4 + (i - 4));
        if (m >= a.M) continue;
#pragma unroll
        for (int h = 0; h < TN / 4; ++h) {
            const int k = n0 + (BN / 2) * h + tn * 4;
            if (k >= a.K) continue;  // K is a multiple of 4: a vector is all in or all out
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float val = acc[i][4 * h + j];
                if (a.alpha) val = val * a.alpha[k + j];
                if (a.bias) val = a.bias[k + j] + val;
                o[j] = val;
            }
            const int off = m * a.K + k;
            if (a.z) {
                const float4 zz = *reinterpret_cast<const float4 *>(a.z + off);
                o[0] += zz.x;
                o[1] += zz.y;
                o[2] += zz.z;
                o[3] += zz.w;
            }
            if (a.relu) {
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = fmaxf(o[j], 0.f);
            }
            *reinterpret_cast<float4 *>(a.y + off) = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

}  // namespace

bool simt_fast_supported(const Dims &d, const void *x, const void *w, const void *y, const void *z) {
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return d.layout == GBCONV_NHWC && d.in_dtype == GBCONV_F32 && d.out_dtype == GBCONV_F32 &&
           d.G == 1 && d.C % 4 == 0 && d.K % 4 == 0 && al(x) && al(w) && al(y) && (!z || al(z)) &&
           (long long)d.N * d.H * d.W * d.C < (1ll << 31) && (d.M() + FM) * d.K < (1ll << 31) &&
           (long long)d.K * d.R * d.S * d.C < (1ll << 31);
}

gbconv_status_t launch_simt_fast_fwd(const Dims &d, const void *x, const void *w, const float *bias,
                                     void *y, cudaStream_t st, const Fused &fz) {
    if (d.M() == 0) return GBCONV_OK;
    FastArgs a;
    a.N = d.N;
    a.C = d.C;
    a.H = d.H;
    a.W = d.W;
    a.K = d.K;
    a.P = d.P;
    a.Q = d.Q;
    a.S = d.S;
    a.RS = d.R * d.S;
    a.u = d.u;
    a.v = d.v;
    a.ph = d.ph;
    a.pw = d.pw;
    a.dh = d.dh;
    a.dw = d.dw;
    a.cb = (d.C + FK - 1) / FK;
    a.ktiles = d.R * d.S * a.cb;
    a.M = (int)d.M();
    a.x = static_cast<const float *>(x);
    a.w = static_cast<const float *>(w);
    a.bias = (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr;
    a.alpha = fz.alpha;
    a.z = static_cast<const float *>(fz.z);
    a.y = static_cast<float *>(y);
    a.relu = (d.flags & GBCONV_FLAG_RELU) ? 1 : 0;
    const long long mt = (d.M() + FM - 1) / FM;
    if (mt > 0x7fffffffll) return GBCONV_ERR_UNSUPPORTED;
    // 64-wide tiles for K <= 64, where 128-wide tiles would not fill one wave
    // of two blocks per SM, and for short reductions (at most 8 k-tiles: each
    // CTA is mostly prologue and epilogue, so more of them per SM pay); the
    // narrow tiles run three per SM
    const long long wide = mt * ((d.K + 127) / 128);
    if (d.K <= 64 || wide < 2LL * sm_count() || a.ktiles <= 8) {
        dim3 grid((unsigned)mt, (unsigned)((d.K + 63) / 64));
        if (grid.y > 65535) return GBCONV_ERR_UNSUPPORTED;
        return cuda_status(launch_pdl(simt_fast_fwd<64, 128>, grid, dim3(128), 0, st, a));
    }
    dim3 grid((unsigned)mt, (unsigned)((d.K + 127) / 128));
    if (grid.y > 65535) return GBCONV_ERR_UNSUPPORTED;
    return cuda_status(launch_pdl(simt_fast_fwd<128, FT>, grid, dim3(FT), 0, st, a));
}

}  // namespace gbc
