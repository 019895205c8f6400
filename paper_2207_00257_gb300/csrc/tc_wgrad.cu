// tc_wgrad.cu -- tensor-core (tcgen05) weight gradient over NHWC BF16 tensors
// (paper Sec. 5.B, backward pass of a convolutional layer):
//
//   dw[k, r, s, c] = sum_{m = (n,p,q)} dy[m, k] * x[n, p*u + r*dh - ph, q*v + s*dw - pw, c]
//
// For one filter tap (r, s) this is a GEMM D[k][c] = sum_m A[k][m] B[c][m]
// with the reduction over output pixels m. Both operands reach shared memory
// "MN-major" (the GEMM's M or N index contiguous, one 128-byte row per
// pixel):
//   A: dy [M][K], one 64-pixel x 64-channel tiled TMA box per 64 output
//      channels (two per 128-channel tile);
//   B: im2col(x) for the tap, the same TMA im2col map as the forward pass
//      with 64-pixel columns, one box per 64 input channels.
// tcgen05.mma (M = 128 output channels, N = C tile, K = 16 pixels) accumulates
// in TMEM. The reduction over N*P*Q is cut into slices; a work unit is
// (slice, output-channel tile, tap, input-channel tile). Each unit's FP32
// partial tile leaves through a 4-D TMA store (clipped at K per slice) into
// the workspace [slice][K][R][S][C]; a second kernel adds the slices in fixed
// order with compensated summation.
//
// Warp roles (288 threads): warps 0 and 6-8 producers (reduction steps taken
// in turn, one box per lane), warp 1 MMA issuer, warps 2-5 epilogue (one TMEM
// lane quarter each). All waits are bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int KT = 128;              // output-channel tile = MMA M
constexpr int PIX = 64;              // pixels per reduction step
constexpr int ATOM = PIX * 128;      // 64 pixel rows x 128 B = one 64-channel block
constexpr int A_STAGE = 2 * ATOM;    // dy for 128 output channels
constexpr int NPROD = 4;             // producer warps: 0 and 6 .. 4 + NPROD
constexpr int NTHREADS = 64 + 32 * 4 + 32 * (NPROD - 1);
constexpr int EPI_WARPS = 4;
constexpr int EPI_BYTES = 8192;      // two 4 KB FP32 chunk buffers per epilogue warp
constexpr int EPI_TOTAL = EPI_WARPS * EPI_BYTES;
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMS_FOR_DEFAULTS = 152;  // split heuristic (host-only, no device query)

struct WgParams {
    CUtensorMap tmG;  // dy [M][K]
    CUtensorMap tmX;  // im2col(x), 64 pixels x 64 channels
    CUtensorMap tmW;  // partials [slices][K][R*S][C], FP32
    int M, P, Q, pw, ph, u, v, dh, dw, S, RS, K;
    int k_tiles, c_tiles, bn, slices, nblocks, units;
    int stages;
    Guard guard;
};

__device__ __forceinline__ void unit_decode(const WgParams &p, int u, int &slice, int &kt, int &rs,
                                            int &ct) {
    ct = u % p.c_tiles;
    int t = u / p.c_tiles;
    rs = t % p.RS;
    t /= p.RS;
    kt = t % p.k_tiles;
    slice = t / p.k_tiles;
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1) tc_wgrad_kernel(const __grid_constant__ WgParams prm) {
    constexpr int B_STAGE = (BN / 64) * ATOM;
    constexpr int TCOLS = 2 * BN;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int stages = prm.stages;
    uint8_t *sA = base;
    uint8_t *sB = base + stages * A_STAGE;
    uint8_t *sEpi = sB + stages * B_STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEpi + EPI_TOTAL);
    uint64_t *full = bars;
    uint64_t *empty = bars + stages;
    uint64_t *tfull = bars + 2 * stages;
    uint64_t *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = prm.guard.wait_ns;

    if (threadIdx.x == 0) {
        for (int i = 0; i < stages; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&tfull[i], 1);
            ptx::mbar_init(&tempty[i], EPI_WARPS);
        }
        ptx::mbar_init(done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, TCOLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (threadIdx.x == 0) {  // descriptors do not depend on earlier kernels
        ptx::prefetch_tmap(&prm.tmG);
        ptx::prefetch_tmap(&prm.tmX);
        ptx::prefetch_tmap(&prm.tmW);
    }
    // Prologue done: now wait for the kernels this one depends on, and let the
    // next kernel on the stream start launching.
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();

    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(prm.guard.err, DEVERR_TIMEOUT);
    };
    auto block_range = [&](int slice, int &b0, int &b1) {
        b0 = (int)((long long)prm.nblocks * slice / prm.slices);
        b1 = (int)((long long)prm.nblocks * (slice + 1) / prm.slices);
    };

    if (warp == 0 || warp >= 6) {
        // ------------------------------ producers ------------------------------
        // The producer warps take the reduction steps (ring stages) in turn;
        // within a step each box is issued by its own lane. On GB300 a TMA load holds
        // its issuing thread about as long as an 8 KB box takes to arrive, so
        // one thread issuing four boxes per step starved the MMAs.
        const unsigned FULL = 0xffffffffu;
        const int me = warp == 0 ? 0 : warp - 5;
        const bool skip = prm.guard.skip_loads != 0;
        constexpr int NBOX = 2 + BN / 64;  // dy: two 64-channel halves; x: BN / 64 blocks
        const uint32_t bytes = A_STAGE + B_STAGE;
        long long it = 0;        // reduction steps of this CTA so far (both warps)
        long long last = -1;     // last step this warp issued
        bool ok = true;
        for (int u = blockIdx.x; ok && u < prm.units; u += gridDim.x) {
            int slice, kt, rs, ct, b0, b1;
            unit_decode(prm, u, slice, kt, rs, ct);
            block_range(slice, b0, b1);
            const int r = rs / prm.S, s = rs - r * prm.S;
            for (int b = b0; b < b1; ++b, ++it) {
                if ((int)(it % NPROD) != me) continue;
                const int stage = (int)(it % stages);
                const uint32_t phase = (uint32_t)((it / stages) & 1);
                int wok = 1;
                if (lane == 0) {
                    wok = ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort_flag);
                    if (wok && !skip) ptx::mbar_arrive_expect_tx(&full[stage], bytes);
                }
                if (!__shfl_sync(FULL, wok, 0)) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                if (skip) continue;
                const int m0 = b * PIX;
                if (lane < 2) {
                    ptx::tma_load_2d(sA + stage * A_STAGE + lane * ATOM, &prm.tmG, &full[stage],
                                     kt * KT + 64 * lane, m0);
                } else if (lane < NBOX) {
                    const int j = lane - 2;
                    const int q = m0 % prm.Q, t = m0 / prm.Q;
                    const int p = t % prm.P, n = t / prm.P;
                    ptx::tma_load_im2col_4d(sB + stage * B_STAGE + j * ATOM, &prm.tmX, &full[stage],
                                            ct * BN + j * 64, q * prm.v - prm.pw, p * prm.u - prm.ph,
                                            n, (uint16_t)(s * prm.dw), (uint16_t)(r * prm.dh));
                }
                last = it;
            }
        }
        // this warp's steps among the last `stages` steps of the CTA are the
        // ones that may still be in flight (an earlier step's slot was reused)
        if (lane == 0) {
            volatile int zero = 0;
            for (long long j = last; j >= 0 && j >= it - stages; j -= NPROD)
                if (!ptx::mbar_wait(&full[(int)(j % stages)], (uint32_t)((j / stages) & 1), lim, &zero))
                    fail();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ----------------------------
            // MN-major operands: 64-element blocks along M / N are 8 KB apart
            // (leading offset); one K step of 16 pixels is 16 rows = 2048 B.
            const uint32_t idesc = ptx::idesc_bf16(BN, 1, 1);
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            for (int u = blockIdx.x; ok && u < prm.units; u += gridDim.x, ++local) {
                int slice, kt, rs, ct, b0, b1;
                unit_decode(prm, u, slice, kt, rs, ct);
                block_range(slice, b0, b1);
                const int acc = local & 1;
                const uint32_t aph = (local >> 1) & 1;
                if (!ptx::mbar_wait(&tempty[acc], aph ^ 1, lim, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int b = b0; b < b1; ++b) {
                    if (!ptx::mbar_wait(&full[stage], phase, lim, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t ad =
                        ptx::sdesc_mnmajor_sw128(ptx::smem_addr(sA + stage * A_STAGE), ATOM);
                    const uint64_t bd =
                        ptx::sdesc_mnmajor_sw128(ptx::smem_addr(sB + stage * B_STAGE), ATOM);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        ptx::mma_f16(d, ad + (uint64_t)(k * 2048 >> 4), bd + (uint64_t)(k * 2048 >> 4),
                                     idesc, (b > b0 || k > 0) ? 1u : 0u);
                    ptx::mma_commit(&empty[stage]);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                ptx::mma_commit(&tfull[acc]);
            }
            ptx::mma_commit(done);
            volatile int zero = 0;
            if (!ptx::mbar_wait(done, 0, lim, &zero)) fail();
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int quarter = warp & 3;
        uint8_t *sbuf = sEpi + (warp - 2) * EPI_BYTES;
        int ebuf = 0;
        int local = 0;
        for (int u = blockIdx.x; u < prm.units; u += gridDim.x, ++local) {
            int slice, kt, rs, ct;
            unit_decode(prm, u, slice, kt, rs, ct);
            const int acc = local & 1;
            const uint32_t aph = (local >> 1) & 1;
            if (!ptx::mbar_wait(&tfull[acc], aph, lim, abort_flag)) {
                fail();
                break;
            }
            ptx::tc_fence_after();
            const int k0 = kt * KT + quarter * 32;
            for (int j = 0; j < BN / 32; ++j) {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(acc * BN + j * 32),
                                        v);
                ptx::tmem_ld_wait();
                if (j == BN / 32 - 1) {
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                }
                if (k0 >= prm.K) continue;
                uint8_t *b = sbuf + ebuf * 4096;
                if (lane == 0) ptx::bulk_wait_read<1>();
                __syncwarp();
                uint8_t *dst = b + lane * 128;  // row = output channel k0 + lane
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4 *>(dst + ((c ^ (lane & 7)) << 4)) =
                        make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    ptx::tma_store_4d(&prm.tmW, b, ct * BN + j * 32, rs, k0, slice);
                    ptx::bulk_commit();
                }
                ebuf ^= 1;
            }
        }
        if (lane == 0) ptx::bulk_wait<0>();
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem_base, TCOLS);
}

int b_stage(int bn) { return (bn / 64) * ATOM; }

int max_stages(int bn) {
    int s = (SMEM_LIMIT - SMEM_ALIGN - BAR_BYTES - EPI_TOTAL) / (A_STAGE + b_stage(bn));
    return std::min(s, 12);
}

size_t smem_bytes(int bn, int stages) {
    return (size_t)SMEM_ALIGN + (size_t)stages * (A_STAGE + b_stage(bn)) + EPI_TOTAL + BAR_BYTES;
}

template <int BN>
gbconv_status_t launch(const WgParams &prm, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_wgrad_kernel<BN>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    return cuda_status(launch_pdl(tc_wgrad_kernel<BN>, dim3(grid), dim3(NTHREADS),
                                  smem_bytes(BN, prm.stages), st, prm));
}

int pick_bn(int C) {
    if (C % 256 == 0) return 256;
    if (C % 128 == 0) return 128;
    return 64;
}

}  // namespace

bool tc_wgrad_supported(const Dims &d) {
    if (d.layout != GBCONV_NHWC || d.in_dtype != GBCONV_BF16) return false;
    if (d.C % 64 || d.K % 8) return false;
    if (d.pw > 127 || d.ph > 127) return false;
    if (d.pw - d.dw * (d.S - 1) < -128 || d.ph - d.dh * (d.R - 1) < -128) return false;
    if (d.u > 8 || d.v > 8) return false;
    if (d.M() >= (1ll << 31)) return false;
    return true;
}

long long tc_wgrad_pixel_steps(const Dims &d) { return (d.M() + PIX - 1) / PIX; }

TcConfig tc_wgrad_default_config(const Dims &d) {
    TcConfig c{};
    c.block_n = pick_bn(d.C);
    c.stages = max_stages(c.block_n);
    const long long per_slice = (long long)((d.K + KT - 1) / KT) * d.R * d.S * (d.C / c.block_n);
    const long long nblocks = (d.M() + PIX - 1) / PIX;
    long long s = per_slice >= SMS_FOR_DEFAULTS ? 1 : SMS_FOR_DEFAULTS / per_slice;
    s = std::min<long long>(s, std::max<long long>(nblocks, 1));
    s = std::min<long long>(s, 256);
    c.split_k = (int)std::max<long long>(s, 1);
    c.raster = 0;
    return c;
}

gbconv_status_t launch_tc_wgrad_partials(const Dims &d, const TcConfig &cfg_in, const void *x,
                                         const void *g, float *ws, cudaStream_t st) {
    TcConfig cfg = cfg_in;
    const int bn = (cfg.block_n == 64 || cfg.block_n == 128 || cfg.block_n == 256) &&
                           d.C % cfg.block_n == 0
                       ? cfg.block_n
                       : pick_bn(d.C);
    const long long nblocks = (d.M() + PIX - 1) / PIX;
    int slices = std::max(1, cfg.split_k);
    if (slices > nblocks) return GBCONV_ERR_INVALID_ARG;  // every slice needs pixels
    // Step `it` is issued by producer warp it % NPROD after its wait on the
    // ring slot's previous use; with fewer slots than producer warps that
    // parity wait could refer to a use two back. Hence stages >= NPROD.
    int stages = cfg.stages >= NPROD && cfg.stages <= max_stages(bn) ? cfg.stages : max_stages(bn);
    WgParams prm;
    memset(&prm, 0, sizeof(prm));
    // dy as [M][K]
    uint64_t gdims[2] = {(uint64_t)d.K, (uint64_t)d.M()};
    uint64_t gstr[1] = {(uint64_t)d.K * 2};
    uint32_t gbox[2] = {64, PIX};
    gbconv_status_t s = encode_tiled(&prm.tmG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g, gdims, gstr,
                                     gbox, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    s = encode_im2col_act(&prm.tmX, d, x, 2, 64, PIX);
    if (s != GBCONV_OK) return s;
    // partials [slices][K][R*S][C], FP32, stored in 32 x 32 chunks
    const int RS = d.R * d.S;
    uint64_t wdims[4] = {(uint64_t)d.C, (uint64_t)RS, (uint64_t)d.K, (uint64_t)slices};
    uint64_t wstr[3] = {(uint64_t)d.C * 4, (uint64_t)RS * d.C * 4, (uint64_t)d.K * RS * d.C * 4};
    uint32_t wbox[4] = {32, 1, 32, 1};
    s = encode_tiled(&prm.tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ws, wdims, wstr, wbox,
                     CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    prm.M = (int)d.M();
    prm.P = d.P;
    prm.Q = d.Q;
    prm.pw = d.pw;
    prm.ph = d.ph;
    prm.u = d.u;
    prm.v = d.v;
    prm.dh = d.dh;
    prm.dw = d.dw;
    prm.S = d.S;
    prm.RS = RS;
    prm.K = d.K;
    prm.k_tiles = (d.K + KT - 1) / KT;
    prm.c_tiles = d.C / bn;
    prm.bn = bn;
    prm.slices = slices;
    prm.nblocks = (int)nblocks;
    prm.units = slices * prm.k_tiles * RS * prm.c_tiles;
    prm.stages = stages;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const int grid = std::min(prm.units, sm_count());
    switch (bn) {
        case 64: return launch<64>(prm, grid, st);
        case 128: return launch<128>(prm, grid, st);
        default: return launch<256>(prm, grid, st);
    }
}

}  // namespace gbc
