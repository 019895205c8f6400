// tc_fwd_shift.cu -- tensor-core forward convolution for stride-1 layers in
// which every filter tap is a row shift of one input band.
//
// Same operation as tc_fwd.cu (forward pass of a convolutional layer, paper
// Sec. 5.B: implicit GEMM D[m, k] = sum_{r,s,c} A[m,(r,s,c)] B[k,(r,s,c)]),
// organised so that each input pixel is fetched once per tile instead of once
// per filter tap:
//
//  * Output pixels of an image are indexed on "extended rows" of Wx columns,
//    Wx a power of two >= Q + (S-1)*dw: e = p*Wx + q. Columns q >= Q are
//    computed and thrown away.
//  * A tile is 128 consecutive extended positions: TR = 128 / Wx whole output
//    rows p0 .. p0+TR-1 of one image.
//  * For each 64-channel (BF16) or 128-channel (FP8) block, one 4-D tiled TMA
//    box loads the band of TR + (R-1)*dh padded input rows, Wx columns each,
//    starting at input (p0 - ph, -pw). Out-of-image pixels read as zeros.
//    Stored row-major with the 128-byte swizzle, band row j = hr*Wx + wc.
//  * The A operand of tap (r, s) is then the 128 band rows starting at row
//    r*dh*Wx + s*dw: the same shared-memory data at a different start
//    address. (tcgen05 applies the swizzle on absolute shared-memory address
//    bits, so any 128-byte row is a valid start.) Garbage columns may read up
//    to (S-1)*dw rows past the band; the stage keeps that much slack.
//  * The filter tiles B[(r,s), c block] stay resident in shared memory when
//    the layer has a single output-channel tile and they fit; otherwise they
//    stream through their own ring.
//  * The epilogue is the one of tc_fwd.cu, storing through a 3-D map of y as
//    [N*P][Q][K] so that garbage columns (q >= Q) are clipped by TMA.
//
// Warp roles and bounded waits as in tc_fwd.cu (320 threads: producer, MMA
// issuer, 8 epilogue warps).
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "epilogue.cuh"
#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int EPI_TOTAL = EPI_TOTAL_BYTES;
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 512;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_SA = 4, MAX_SB = 12;

struct ShiftParams {
    CUtensorMap tmX;  // x [N][H][W][C], box {KE, Wx, nr, 1}
    CUtensorMap tmB;  // w [K][R*S][C], box {KE, 1, bn}
    CUtensorMap tmY;  // y [N*P][Q][K], box {32, 32, 1}
    int N, P, Q;
    int pw, ph, dh, dw, S, RS;
    int wx_log2, TR;
    int c_blocks, bn, n_tiles, p_tiles, num_tiles;
    int band_bytes, band_stride, b_resident, stages_a, stages_b;
    int raster;
    EpiArgs epi;
    const float *x_scale;
    Guard guard;
};

__device__ __forceinline__ void sdecode(const ShiftParams &p, int tile, int &n, int &p0, int &nt) {
    const int mts = p.N * p.p_tiles;
    int mt;
    if (p.raster == 0) {
        mt = tile / p.n_tiles;
        nt = tile - mt * p.n_tiles;
    } else {
        nt = tile / mts;
        mt = tile - nt * mts;
    }
    n = mt / p.p_tiles;
    p0 = (mt - n * p.p_tiles) * p.TR;
}

// FUSED: the epilogue also applies the per-channel scale and the residual.
template <int BN, bool FP8, bool FUSED>
__global__ void __launch_bounds__(EpiShape<BN>::threads, 1)
    tc_fwd_shift_kernel(const __grid_constant__ ShiftParams prm) {
    constexpr int EPI_WARPS = EpiShape<BN>::warps;
    constexpr int EPI_BYTES = EpiShape<BN>::warp_bytes;
    constexpr int EPI_GROUPS = EPI_WARPS / 4;  // warps per TMEM lane quarter
    constexpr int KE = FP8 ? 128 : 64;
    constexpr int TCOLS = (2 * BN < 32) ? 32 : 2 * BN;
    constexpr int B_TILE = BN * 128;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int SA = prm.stages_a, SB = prm.stages_b;
    const int b_slots = prm.b_resident ? prm.RS * prm.c_blocks : SB;
    uint8_t *sA = base;
    uint8_t *sB = sA + SA * prm.band_stride;
    uint8_t *sEpi = sB + b_slots * B_TILE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEpi + EPI_TOTAL);
    uint64_t *fullA = bars;               // [SA]
    uint64_t *emptyA = fullA + MAX_SA;    // [SA]
    uint64_t *fullB = emptyA + MAX_SA;    // [SB] (slot 0 only when resident)
    uint64_t *emptyB = fullB + MAX_SB;    // [SB]
    uint64_t *tfull = emptyB + MAX_SB;    // [2]
    uint64_t *tempty = tfull + 2;         // [2]
    uint64_t *done = tempty + 2;          // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = prm.guard.wait_ns;

    if (threadIdx.x == 0) {
        for (int i = 0; i < SA; ++i) {
            ptx::mbar_init(&fullA[i], 1);
            ptx::mbar_init(&emptyA[i], 1);
        }
        for (int i = 0; i < (prm.b_resident ? 1 : SB); ++i) {
            ptx::mbar_init(&fullB[i], 1);
            ptx::mbar_init(&emptyB[i], 1);
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
        ptx::prefetch_tmap(&prm.tmX);
        ptx::prefetch_tmap(&prm.tmB);
        ptx::prefetch_tmap(&prm.tmY);
    }
    // Prologue done: now wait for the kernels this one depends on, and let the
    // next kernel on the stream start launching.
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();

    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(prm.guard.err, DEVERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------ producer ------------------------------
            const bool skip = prm.guard.skip_loads != 0;
            bool ok = true;
            int issued_b = 0;  // resident filter: 1 after its load was issued
            if (prm.b_resident && !skip) {
                ptx::mbar_arrive_expect_tx(&fullB[0], (uint32_t)(prm.RS * prm.c_blocks * B_TILE));
                for (int cb = 0; cb < prm.c_blocks; ++cb)
                    for (int t = 0; t < prm.RS; ++t)
                        ptx::tma_load_3d(sB + (cb * prm.RS + t) * B_TILE, &prm.tmB, &fullB[0],
                                         cb * KE, t, 0);
                issued_b = 1;
            }
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            int issued_a = 0, issued_bs = 0;
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x) {
                int n, p0, nt;
                sdecode(prm, tile, n, p0, nt);
                for (int cb = 0; ok && cb < prm.c_blocks; ++cb) {
                    if (!ptx::mbar_wait(&emptyA[sa], pa ^ 1, lim, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (!skip) {
                        ptx::mbar_arrive_expect_tx(&fullA[sa], (uint32_t)prm.band_bytes);
                        ptx::tma_load_4d(sA + sa * prm.band_stride, &prm.tmX, &fullA[sa], cb * KE,
                                         -prm.pw, p0 - prm.ph, n);
                        ++issued_a;
                    }
                    if (++sa == SA) {
                        sa = 0;
                        pa ^= 1;
                    }
                    if (prm.b_resident) continue;
                    for (int t = 0; t < prm.RS; ++t) {
                        if (!ptx::mbar_wait(&emptyB[sb], pb ^ 1, lim, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        if (!skip) {
                            ptx::mbar_arrive_expect_tx(&fullB[sb], (uint32_t)B_TILE);
                            ptx::tma_load_3d(sB + sb * B_TILE, &prm.tmB, &fullB[sb], cb * KE, t,
                                             nt * prm.bn);
                            ++issued_bs;
                        }
                        if (++sb == SB) {
                            sb = 0;
                            pb ^= 1;
                        }
                    }
                }
            }
            // Drain every copy still in flight before shared memory is released.
            volatile int zero = 0;
            {
                int st = sa;
                uint32_t ph = pa;
                for (int i = 0; i < min(issued_a, SA); ++i) {
                    if (st == 0) {
                        st = SA;
                        ph ^= 1;
                    }
                    --st;
                    if (!ptx::mbar_wait(&fullA[st], ph, lim, &zero)) fail();
                }
            }
            {
                int st = sb;
                uint32_t ph = pb;
                for (int i = 0; i < min(issued_bs, SB); ++i) {
                    if (st == 0) {
                        st = SB;
                        ph ^= 1;
                    }
                    --st;
                    if (!ptx::mbar_wait(&fullB[st], ph, lim, &zero)) fail();
                }
            }
            if (issued_b && !ptx::mbar_wait(&fullB[0], 0, lim, &zero)) fail();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ----------------------------
            bool ok = true;
            if (prm.b_resident) {
                if (!ptx::mbar_wait(&fullB[0], 0, lim, abort_flag)) {
                    fail();
                    ok = false;
                }
            }
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            int local = 0;
            const uint32_t idesc = FP8 ? ptx::idesc_e4m3(prm.bn) : ptx::idesc_bf16(prm.bn);
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x, ++local) {
                const int acc = local & 1;
                const uint32_t aph = (local >> 1) & 1;
                if (!ptx::mbar_wait(&tempty[acc], aph ^ 1, lim, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int cb = 0; ok && cb < prm.c_blocks; ++cb) {
                    if (!ptx::mbar_wait(&fullA[sa], pa, lim, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t a_base = ptx::smem_addr(sA + sa * prm.band_stride);
                    int r = 0, s = 0;
                    for (int t = 0; t < prm.RS; ++t) {
                        uint32_t b_addr;
                        if (prm.b_resident) {
                            b_addr = ptx::smem_addr(sB + (cb * prm.RS + t) * B_TILE);
                        } else {
                            if (!ptx::mbar_wait(&fullB[sb], pb, lim, abort_flag)) {
                                fail();
                                ok = false;
                                break;
                            }
                            ptx::tc_fence_after();
                            b_addr = ptx::smem_addr(sB + sb * B_TILE);
                        }
                        const uint32_t shift = (uint32_t)(((r * prm.dh) << prm.wx_log2) + s * prm.dw);
                        const uint64_t ad = ptx::sdesc_kmajor_sw128(a_base + shift * 128u);
                        const uint64_t bd = ptx::sdesc_kmajor_sw128(b_addr);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t accum = (cb | t | k) != 0;
                            if (FP8)
                                ptx::mma_f8(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                            else
                                ptx::mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                        }
                        if (!prm.b_resident) {
                            ptx::mma_commit(&emptyB[sb]);
                            if (++sb == SB) {
                                sb = 0;
                                pb ^= 1;
                            }
                        }
                        if (++s == prm.S) {
                            s = 0;
                            ++r;
                        }
                    }
                    if (!ok) break;
                    ptx::mma_commit(&emptyA[sa]);
                    if (++sa == SA) {
                        sa = 0;
                        pa ^= 1;
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
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        uint8_t *sbuf = sEpi + ew * EPI_BYTES;
        int ebuf = 0;
        int local = 0;
        const int wx_mask = (1 << prm.wx_log2) - 1;
        for (int tile = blockIdx.x; tile < prm.num_tiles; tile += gridDim.x, ++local) {
            int n, p0, nt;
            sdecode(prm, tile, n, p0, nt);
            const int acc = local & 1;
            const uint32_t aph = (local >> 1) & 1;
            const int p = p0 + ((quarter * 32) >> prm.wx_log2);
            const int q0 = (quarter * 32) & wx_mask;
            const bool rows_ok = p < prm.P && q0 < prm.Q;
            if constexpr (FUSED) {  // residual rows into L2, this tile (first) and the next
                if (prm.epi.z)
                    for (int t2 = (local == 0 ? tile : tile + (int)gridDim.x);
                         t2 <= tile + (int)gridDim.x && t2 < prm.num_tiles; t2 += (int)gridDim.x) {
                        int n2, p02, nt2;
                        sdecode(prm, t2, n2, p02, nt2);
                        const int pp = p02 + ((quarter * 32) >> prm.wx_log2);
                        const int qq = (quarter * 32) & wx_mask;
                        if (pp < prm.P && qq < prm.Q)
                            for (int j = half; j < prm.bn / 32; j += EPI_GROUPS)
                                prefetch_residual(prm.epi, nt2 * prm.bn + j * 32, qq, n2 * prm.P + pp,
                                                  lane);
                    }
            }
            if (!ptx::mbar_wait(&tfull[acc], aph, lim, abort_flag)) {
                fail();
                break;
            }
            ptx::tc_fence_after();
            const float xs = FP8 ? __ldg(prm.x_scale) : 1.f;
            const int nchunks = prm.bn / 32;
            bool released = false;
            for (int j = half; j < nchunks; j += EPI_GROUPS) {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(acc * BN + j * 32),
                                        v);
                ptx::tmem_ld_wait();
                if (j + EPI_GROUPS >= nchunks) {
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                    released = true;
                }
                const int col0 = nt * prm.bn + j * 32;
                if (!rows_ok || col0 >= prm.epi.K) continue;
                epilogue_chunk<FP8, EpiShape<BN>::nbuf, FUSED>(v, prm.epi, &prm.tmY, xs, col0, q0, n * prm.P + p, lane, sbuf,
                                    ebuf);
            }
            if (!released) {
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
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

struct Plan {
    int wx_log2, TR, nr, band_bytes, band_stride, c_blocks, b_resident, stages_a, stages_b;
};

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Shared-memory plan of the shifted-band kernel for tile width bn (false if
// the layer does not suit it).
bool make_plan(const Dims &d, int bn, Plan *pl) {
    if (d.u != 1 || d.v != 1) return false;
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    const int ke = fp8 ? 128 : 64;
    const int need = d.Q + (d.S - 1) * d.dw;
    int wx = 32;
    while (wx < need) wx *= 2;
    if (wx > 128) return false;
    Plan p{};
    p.wx_log2 = ilog2(wx);
    p.TR = 128 / wx;
    p.nr = p.TR + (d.R - 1) * d.dh;
    if (p.nr > 256) return false;
    p.band_bytes = 128 * wx * p.nr;
    const int slack = (d.S - 1) * d.dw * 128;
    p.band_stride = (p.band_bytes + slack + 1023) / 1024 * 1024;
    if (p.band_stride > 64 * 1024) return false;
    p.c_blocks = (d.C + ke - 1) / ke;
    const int budget = SMEM_LIMIT - SMEM_ALIGN - BAR_BYTES - EPI_TOTAL;
    const int btile = bn * 128;
    const long long b_total = (long long)d.R * d.S * p.c_blocks * btile;
    const int n_tiles = (d.K + bn - 1) / bn;
    if (n_tiles == 1 && b_total + 2ll * p.band_stride <= budget) {
        p.b_resident = 1;
        p.stages_a = (int)std::min<long long>(MAX_SA, (budget - b_total) / p.band_stride);
        p.stages_b = 0;
    } else {
        p.b_resident = 0;
        p.stages_a = 2;
        p.stages_b = std::min(MAX_SB, (budget - 2 * p.band_stride) / btile);
        if (p.stages_b < 2) return false;
        if (p.stages_b >= 8 && budget - 3 * p.band_stride >= 8 * btile) p.stages_a = 3;
        p.stages_b = std::min(MAX_SB, (budget - p.stages_a * p.band_stride) / btile);
    }
    *pl = p;
    return true;
}

size_t smem_bytes(const Dims &d, int bn, const Plan &p) {
    const int b_slots = p.b_resident ? d.R * d.S * p.c_blocks : p.stages_b;
    return (size_t)SMEM_ALIGN + (size_t)p.stages_a * p.band_stride + (size_t)b_slots * bn * 128 +
           EPI_TOTAL + BAR_BYTES;
}

template <int BN, bool FP8, bool FUSED>
gbconv_status_t launch_one(const ShiftParams &prm, size_t smem, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fwd_shift_kernel<BN, FP8, FUSED>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    return cuda_status(launch_pdl(tc_fwd_shift_kernel<BN, FP8, FUSED>, dim3(grid),
                                  dim3(EpiShape<BN>::threads), smem, st, prm));
}

template <int BN, bool FP8>
gbconv_status_t launch(const ShiftParams &prm, size_t smem, int grid, cudaStream_t st) {
    return (prm.epi.alpha || prm.epi.z) ? launch_one<BN, FP8, true>(prm, smem, grid, st)
                                        : launch_one<BN, FP8, false>(prm, smem, grid, st);
}

}  // namespace

bool tc_fwd_shift_supported(const Dims &d, int block_n) {
    Plan p;
    return tc_fwd_supported(d) && make_plan(d, block_n, &p);
}

bool tc_fwd_shift_preferred(const Dims &d, int block_n) {
    // Measured on GB300: the band kernel wins when the whole filter stays in
    // shared memory; when the filter streams, the im2col kernel's deeper
    // combined ring is faster.
    Plan p;
    return tc_fwd_supported(d) && make_plan(d, block_n, &p) && p.b_resident;
}

gbconv_status_t launch_tc_fwd_shift(const Dims &d, const TcConfig &cfg, const void *x,
                                    const void *w, const float *bias, const float *x_scale,
                                    const float *w_scale, void *y, cudaStream_t st,
                                    const Fused &fz) {
    const int bn = cfg.block_n;
    if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return GBCONV_ERR_INVALID_ARG;
    Plan pl;
    if (!make_plan(d, bn, &pl)) return GBCONV_ERR_UNSUPPORTED;
    if (d.M() == 0) return GBCONV_OK;
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    const int eb = fp8 ? 1 : 2, ke = 128 / eb;
    const CUtensorMapDataType in_t =
        fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    ShiftParams prm;
    memset(&prm, 0, sizeof(prm));
    // x [N][H][W][C]: one band of nr rows x Wx columns per load
    uint64_t xd[4] = {(uint64_t)d.C, (uint64_t)d.W, (uint64_t)d.H, (uint64_t)d.N};
    uint64_t xs[3] = {(uint64_t)d.C * eb, (uint64_t)d.W * d.C * eb, (uint64_t)d.H * d.W * d.C * eb};
    uint32_t xb[4] = {(uint32_t)ke, (uint32_t)(1 << pl.wx_log2), (uint32_t)pl.nr, 1};
    gbconv_status_t s = encode_tiled(&prm.tmX, in_t, 4, x, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    uint64_t wd[3] = {(uint64_t)d.C, (uint64_t)d.R * d.S, (uint64_t)d.K};
    uint64_t wstr[2] = {(uint64_t)d.C * eb, (uint64_t)d.R * d.S * d.C * eb};
    uint32_t wbx[3] = {(uint32_t)ke, 1, (uint32_t)bn};
    s = encode_tiled(&prm.tmB, in_t, 3, w, wd, wstr, wbx, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    const bool of32 = d.out_dtype == GBCONV_F32;
    uint64_t yd[3] = {(uint64_t)d.K, (uint64_t)d.Q, (uint64_t)d.N * d.P};
    uint64_t ys[2] = {(uint64_t)d.K * (of32 ? 4 : 2), (uint64_t)d.Q * d.K * (of32 ? 4 : 2)};
    uint32_t yb[3] = {32, 32, 1};
    s = encode_tiled(&prm.tmY, of32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     3, y, yd, ys, yb, of32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
    if (s != GBCONV_OK) return s;
    prm.N = d.N;
    prm.P = d.P;
    prm.Q = d.Q;
    prm.pw = d.pw;
    prm.ph = d.ph;
    prm.dh = d.dh;
    prm.dw = d.dw;
    prm.S = d.S;
    prm.RS = d.R * d.S;
    prm.wx_log2 = pl.wx_log2;
    prm.TR = pl.TR;
    prm.c_blocks = pl.c_blocks;
    prm.bn = bn;
    prm.n_tiles = (d.K + bn - 1) / bn;
    prm.p_tiles = (d.P + pl.TR - 1) / pl.TR;
    const long long tiles = (long long)d.N * prm.p_tiles * prm.n_tiles;
    if (tiles >= (1ll << 31)) return GBCONV_ERR_UNSUPPORTED;
    prm.num_tiles = (int)tiles;
    prm.band_bytes = pl.band_bytes;
    prm.band_stride = pl.band_stride;
    prm.b_resident = pl.b_resident;
    prm.stages_a = pl.stages_a;
    prm.stages_b = pl.stages_b;
    prm.raster = cfg.raster;
    prm.epi = EpiArgs{d.K, (d.flags & GBCONV_FLAG_RELU) ? 1 : 0, of32 ? 1 : 0,
                      (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr, w_scale, fz.alpha, fz.z,
                      d.M(), d.Q};
    prm.x_scale = x_scale;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const size_t smem = smem_bytes(d, bn, pl);
    const int grid = std::min(prm.num_tiles, sm_count());
    switch (bn) {
        case 32: return fp8 ? launch<32, true>(prm, smem, grid, st) : launch<32, false>(prm, smem, grid, st);
        case 64: return fp8 ? launch<64, true>(prm, smem, grid, st) : launch<64, false>(prm, smem, grid, st);
        case 128: return fp8 ? launch<128, true>(prm, smem, grid, st) : launch<128, false>(prm, smem, grid, st);
        default: return fp8 ? launch<256, true>(prm, smem, grid, st) : launch<256, false>(prm, smem, grid, st);
    }
}

}  // namespace gbc
