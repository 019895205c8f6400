// tc_fwd.cu -- tensor-core (tcgen05) implicit-GEMM forward convolution over
// NHWC, BF16 or FP8-E4M3 operands, FP32 accumulation in Tensor Memory.
//
// The forward pass of a convolutional layer (paper Sec. 5.B, which performs
// it as im2col followed by a GEMM) is computed here as an implicit GEMM:
//   D[m, k] = sum_{(r,s,c)} A[m, (r,s,c)] * B[k, (r,s,c)]
// with m = (n, p, q) an output pixel, A the im2col matrix of x (never
// materialised: a TMA im2col-mode load produces one 128-pixel x 128-byte
// tile of it per filter tap and channel block) and B the KRSC filter.
//
// One persistent CTA per SM walks output tiles of 128 pixels x BN channels.
// Warp roles (320 threads):
//   warp 0  producer: one thread issues the TMA loads of A (im2col, or plain
//           tiled rows for 1x1 stride-1 unpadded layers) and B (tiled) into an
//           S-stage shared-memory ring ("full"/"empty" mbarriers);
//   warp 1  MMA issuer: one thread issues tcgen05.mma (128 x BN x 16 for BF16,
//           x 32 for E4M3) into one of two TMEM accumulators and commits each
//           stage back to the producer;
//   warps 2-9 epilogue: two warps per TMEM lane quarter, alternating 32-column
//           chunks: tcgen05.ld, FP8 scales and bias (one coalesced load, then
//           warp shuffles), ReLU, conversion, a swizzled staging buffer in
//           shared memory and a TMA tensor store of the 32 x 32 chunk. A warp
//           releases the accumulator right after its last TMEM load, so the
//           MMA warp refills it while the stores drain.
// Every mbarrier wait is bounded (ptx::mbar_wait); on a timeout the kernel
// records DEVERR_TIMEOUT, drains its own in-flight copies and MMAs, frees
// TMEM and returns.
//
// The same kernel body serves the grouped launch: G problems, each with its
// own tensor maps and sizes in the kernel parameters, share one tile space.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "epilogue.cuh"
#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int BM = 128;
constexpr int A_BYTES = BM * 128;  // 128 pixels x 128 bytes of channels
constexpr int EPI_TOTAL = EPI_TOTAL_BYTES;
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 1024;
constexpr int ZMAX = 4;  // fused residual: TMA-loaded chunks per epilogue warp and tile
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int GMAX = 64;  // problems per grouped launch

struct ProbArgs {
    int M, P, Q;
    int pw, ph, u, v, dh, dw, S, RS;
    int c_blocks, kb_per_tile;
    int n_tiles, bn, K;
    int relu, out_f32, a_tiled;
    const float *bias;
    const float *x_scale;
    const float *w_scale;
};

template <int G>
struct FwdParams {
    CUtensorMap tmA[G];
    CUtensorMap tmB[G];
    CUtensorMap tmY[G];
    ProbArgs pa[G];
    int tile_start[G + 1];  // prefix sums of tiles per problem
    int count;
    int num_tiles;
    int stages;
    int raster;
    const float *alpha;  // fused epilogue of a single problem (G == 1): per-channel scale
    const void *z;       // and residual; null otherwise
    CUtensorMap tmZ;     // residual as y's store map (BF16 output): loaded into the staging
    int z_tma;           // buffers by TMA ahead of the accumulator when set
    Guard guard;
};

// All per-problem descriptors of a grouped launch travel as kernel parameters
// (no host-to-device copy, graph-capturable): they must fit the 32764-byte
// parameter limit.
static_assert(sizeof(FwdParams<GMAX>) <= 32764, "grouped kernel parameters too large");

template <int BN>
struct TmemCols {
    static constexpr int v = (2 * BN < 32) ? 32 : 2 * BN;
};

template <int G>
__device__ __forceinline__ void decode(const FwdParams<G> &prm, int tile, int &g, int &mt,
                                       int &nt) {
    g = 0;
    if (G > 1) {
        while (g + 1 < prm.count && tile >= prm.tile_start[g + 1]) ++g;
    }
    const int lt = tile - prm.tile_start[g];
    const int nts = prm.pa[g].n_tiles;
    if (prm.raster == 0) {
        mt = lt / nts;
        nt = lt - mt * nts;
    } else {
        const int mts = (prm.pa[g].M + BM - 1) / BM;
        nt = lt / mts;
        mt = lt - nt * mts;
    }
}

// FMODE (single-problem launches only): 0 plain epilogue; 1 fused per-channel
// scale and residual read by the epilogue threads (FP32 output, or no
// residual); 2 fused with the residual tiles brought into the staging
// buffers by TMA ahead of the accumulator (BF16 output).
template <int BN, bool FP8, int G, int FMODE = 0>
__global__ void __launch_bounds__(EpiShape<BN>::threads, 1) tc_fwd_kernel(const __grid_constant__ FwdParams<G> prm) {
    constexpr bool FUSED = FMODE != 0;
    constexpr bool ZT = FMODE == 2;
    constexpr int EPI_WARPS = EpiShape<BN>::warps;
    constexpr int EPI_BYTES = EpiShape<BN>::warp_bytes;
    constexpr int EPI_GROUPS = EPI_WARPS / 4;  // warps per TMEM lane quarter
    constexpr int KE = FP8 ? 128 : 64;         // reduction elements per 128-byte row
    constexpr int KSTEPS = 4;                  // 4 MMAs of 32 bytes of K per row
    constexpr int TCOLS = TmemCols<BN>::v;
    constexpr int B_STAGE = BN * 128;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int stages = prm.stages;
    uint8_t *sA = base;
    uint8_t *sB = base + stages * A_BYTES;
    uint8_t *sEpi = sB + stages * B_STAGE;  // 1024-aligned: A and B stages are multiples of 1024
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEpi + EPI_TOTAL);
    uint64_t *full = bars;                // [stages]
    uint64_t *empty = bars + stages;      // [stages]
    uint64_t *tfull = bars + 2 * stages;  // [2]
    uint64_t *tempty = tfull + 2;         // [2]
    uint64_t *done = tempty + 2;          // [1]
    uint64_t *zbar = done + 1;            // [EPI_WARPS][ZMAX] fused residual loads
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(zbar + EPI_WARPS * ZMAX);
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
        if (FUSED)
            for (int i = 0; i < EPI_WARPS * ZMAX; ++i) ptx::mbar_init(&zbar[i], 1);
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
    // Tensor-map descriptors do not depend on earlier kernels: fetch them
    // while the previous kernel drains.
    if (warp == 0)
        for (int g = lane; g < prm.count; g += 32) {
            ptx::prefetch_tmap(&prm.tmA[g]);
            ptx::prefetch_tmap(&prm.tmB[g]);
            ptx::prefetch_tmap(&prm.tmY[g]);
        }
    // The first tile's operand boxes into L2 while the previous kernel
    // drains. A prefetch moves nothing into shared memory or registers, and L2
    // stays coherent with the previous kernel's writes, so it is safe before
    // the dependency wait; the loads themselves come after it.
    if (threadIdx.x == 0 && (int)blockIdx.x < prm.num_tiles) {
        int g, mt, nt;
        decode(prm, blockIdx.x, g, mt, nt);
        const ProbArgs &pa = prm.pa[g];
        const int m0 = mt * BM;
        const int q = m0 % pa.Q, t = m0 / pa.Q;
        const int p = t % pa.P, n = t / pa.P;
        const int wc = q * pa.v - pa.pw, hc = p * pa.u - pa.ph;
        int r = 0, s = 0;
        for (int rs = 0; rs < pa.RS; ++rs) {
            for (int cb = 0; cb < pa.c_blocks; ++cb) {
                if (pa.a_tiled)
                    ptx::tma_prefetch_2d(&prm.tmA[g], cb * KE, m0);
                else
                    ptx::tma_prefetch_im2col_4d(&prm.tmA[g], cb * KE, wc, hc, n,
                                                (uint16_t)(s * pa.dw), (uint16_t)(r * pa.dh));
                ptx::tma_prefetch_3d(&prm.tmB[g], cb * KE, rs, nt * pa.bn);
            }
            if (++s == pa.S) {
                s = 0;
                ++r;
            }
        }
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
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x) {
                int g, mt, nt;
                decode(prm, tile, g, mt, nt);
                const ProbArgs &pa = prm.pa[g];
                const int m0 = mt * BM;
                const int q = m0 % pa.Q, t = m0 / pa.Q;
                const int p = t % pa.P, n = t / pa.P;
                const int wc = q * pa.v - pa.pw, hc = p * pa.u - pa.ph;
                const int n0 = nt * pa.bn;
                const CUtensorMap *ta = &prm.tmA[g];
                const CUtensorMap *tb = &prm.tmB[g];
                const uint32_t bytes = A_BYTES + pa.bn * 128;
                int r = 0, s = 0;
                for (int rs = 0; ok && rs < pa.RS; ++rs) {
                    for (int cb = 0; cb < pa.c_blocks; ++cb) {
                        if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        if (!prm.guard.skip_loads) {
                            ptx::mbar_arrive_expect_tx(&full[stage], bytes);
                            if (pa.a_tiled)
                                ptx::tma_load_2d(sA + stage * A_BYTES, ta, &full[stage], cb * KE, m0);
                            else
                                ptx::tma_load_im2col_4d(sA + stage * A_BYTES, ta, &full[stage],
                                                        cb * KE, wc, hc, n, (uint16_t)(s * pa.dw),
                                                        (uint16_t)(r * pa.dh));
                            ptx::tma_load_3d(sB + stage * B_STAGE, tb, &full[stage], cb * KE, rs,
                                             n0);
                            ++issued;
                        }
                        if (++stage == stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (++s == pa.S) {
                        s = 0;
                        ++r;
                    }
                }
            }
            // Drain: the last min(issued, stages) fills must have landed before
            // this CTA's shared memory can be released.
            int st = stage;
            uint32_t ph = phase;
            for (int i = 0; i < min(issued, stages); ++i) {
                if (st == 0) {
                    st = stages;
                    ph ^= 1;
                }
                --st;
                if (!ptx::mbar_wait(&full[st], ph, lim, abort_flag)) {
                    // give the copy one more full period without the abort shortcut
                    volatile int zero = 0;
                    if (!ptx::mbar_wait(&full[st], ph, lim, &zero)) fail();
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ----------------------------
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x, ++local) {
                int g, mt, nt;
                decode(prm, tile, g, mt, nt);
                const ProbArgs &pa = prm.pa[g];
                const int acc = local & 1;
                const uint32_t aph = (local >> 1) & 1;
                if (!ptx::mbar_wait(&tempty[acc], aph ^ 1, lim, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                const uint32_t idesc = FP8 ? ptx::idesc_e4m3(pa.bn) : ptx::idesc_bf16(pa.bn);
                for (int kb = 0; kb < pa.kb_per_tile; ++kb) {
                    if (!ptx::mbar_wait(&full[stage], phase, lim, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t ad = ptx::sdesc_kmajor_sw128(ptx::smem_addr(sA + stage * A_BYTES));
                    const uint64_t bd = ptx::sdesc_kmajor_sw128(ptx::smem_addr(sB + stage * B_STAGE));
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k) {
                        // +32 bytes of K per step: +2 in the descriptor's address field
                        if (FP8)
                            ptx::mma_f8(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                        else
                            ptx::mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
                    }
                    ptx::mma_commit(&empty[stage]);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                ptx::mma_commit(&tfull[acc]);
            }
            // Drain: every MMA this thread issued must be complete before TMEM is freed.
            ptx::mma_commit(done);
            volatile int zero = 0;
            if (!ptx::mbar_wait(done, 0, lim, &zero)) fail();
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int ew = warp - 2;        // 0..7
        const int quarter = warp & 3;   // TMEM lanes this warp may access
        const int half = ew >> 2;       // this warp takes chunks j with j % EPI_GROUPS == half
        uint8_t *sbuf = sEpi + ew * EPI_BYTES;
        int ebuf = 0;
        int local = 0;
        uint32_t zbits = 0;  // phase of each residual slot's barrier
        uint32_t zdrain = 0, zdpar = 0;  // slots (and phases) an abort left in flight
        for (int tile = blockIdx.x; tile < prm.num_tiles; tile += gridDim.x, ++local) {
            int g, mt, nt;
            decode(prm, tile, g, mt, nt);
            const ProbArgs &pa = prm.pa[g];
            const int acc = local & 1;
            const uint32_t aph = (local >> 1) & 1;
            uint32_t zmask = 0, zpar = 0;  // residual slots loaded for this tile, their phases
            if constexpr (FUSED && G == 1) {
                if (ZT) {
                    // residual chunks of this warp -> its staging buffers, by TMA, while
                    // the MMAs run (the buffers' previous stores must have been read)
                    if (lane == 0) {
                        // the next tile's residual chunks into L2 meanwhile
                        const int t2 = tile + (int)gridDim.x;
                        if (t2 < prm.num_tiles) {
                            int g2, mt2, nt2;
                            decode(prm, t2, g2, mt2, nt2);
                            for (int j = half; j < pa.bn / 32; j += EPI_GROUPS) {
                                const int c0z = nt2 * pa.bn + j * 32, r0z = mt2 * BM + quarter * 32;
                                if (c0z < pa.K && r0z < pa.M) ptx::tma_prefetch_2d(&prm.tmZ, c0z, r0z);
                            }
                        }
                        ptx::bulk_wait_read<0>();
                    }
                    for (int j = half, ci = 0; j < pa.bn / 32; j += EPI_GROUPS, ++ci) {
                        const int c0z = nt * pa.bn + j * 32, r0z = mt * BM + quarter * 32;
                        if (c0z >= pa.K || r0z >= pa.M) continue;
                        zmask |= 1u << ci;
                        if (lane == 0) {
                            ptx::mbar_arrive_expect_tx(&zbar[ew * ZMAX + ci], 2048);
                            ptx::tma_load_2d(sbuf + ci * 2048, &prm.tmZ, &zbar[ew * ZMAX + ci], c0z,
                                             r0z);
                        }
                    }
                    zpar = zbits;
                    zbits ^= zmask;
                    __syncwarp();
                } else if (prm.z) {
                    // residual rows of this warp's chunks into L2, one tile ahead (the
                    // first tile's at the start): they arrive while the MMAs run
                    const EpiArgs ea{pa.K, 0, pa.out_f32, nullptr, nullptr, nullptr, prm.z,
                                     (long long)pa.M, pa.Q};
                    for (int t2 = (local == 0 ? tile : tile + (int)gridDim.x);
                         t2 <= tile + (int)gridDim.x && t2 < prm.num_tiles; t2 += (int)gridDim.x) {
                        int g2, mt2, nt2;
                        decode(prm, t2, g2, mt2, nt2);
                        for (int j = half; j < pa.bn / 32; j += EPI_GROUPS)
                            prefetch_residual(ea, nt2 * pa.bn + j * 32, mt2 * BM + quarter * 32, -1,
                                              lane);
                    }
                }
            }

            if (!ptx::mbar_wait(&tfull[acc], aph, lim, abort_flag)) {
                fail();
                zdrain = zmask;  // residual loads of this tile still to land
                zdpar = zpar;
                break;
            }
            ptx::tc_fence_after();
            const int row0 = mt * BM + quarter * 32;
            const float xs = FP8 ? __ldg(pa.x_scale) : 1.f;
            const int nchunks = pa.bn / 32;
            bool released = false;
            for (int j = half; j < nchunks; j += EPI_GROUPS) {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(acc * BN + j * 32),
                                        v);
                ptx::tmem_ld_wait();
                if (j + EPI_GROUPS >= nchunks) {  // last TMEM read of this warp for this tile
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                    released = true;
                }
                const int col0 = nt * pa.bn + j * 32;
                if (col0 >= pa.K || row0 >= pa.M) continue;  // chunk entirely outside y
                const EpiArgs ea{pa.K, pa.relu, pa.out_f32, pa.bias, pa.w_scale,
                                 G == 1 ? prm.alpha : nullptr, G == 1 ? prm.z : nullptr,
                                 (long long)pa.M, pa.Q};
                if constexpr (ZT) {
                    const int ci = (j - half) / EPI_GROUPS;
                    if (!((zmask >> ci) & 1u)) continue;
                    if (!ptx::mbar_wait(&zbar[ew * ZMAX + ci], (zpar >> ci) & 1u, lim, abort_flag)) {
                        fail();
                        continue;
                    }
                    epilogue_chunk_zsmem<FP8>(v, ea, &prm.tmY[g], xs, col0, row0, -1, lane,
                                              sbuf + ci * 2048);
                } else {
                    epilogue_chunk<FP8, EpiShape<BN>::nbuf, FUSED>(v, ea, &prm.tmY[g], xs, col0, row0,
                                                                   -1, lane, sbuf, ebuf);
                }
            }
            if (!released) {
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
            }
        }
        if (FUSED && zdrain && lane == 0) {
            // an aborted tile's residual loads must land before the CTA leaves
            volatile int zero = 0;
            for (int ci = 0; ci < ZMAX; ++ci)
                if ((zdrain >> ci) & 1u) ptx::mbar_wait(&zbar[ew * ZMAX + ci], (zdpar >> ci) & 1u, lim, &zero);
        }
        if (lane == 0) ptx::bulk_wait<0>();  // stores done before the CTA leaves
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem_base, TCOLS);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int BN>
constexpr int b_stage_bytes() { return BN * 128; }

int max_stages(int bn) {
    int per = A_BYTES + bn * 128;
    int s = (SMEM_LIMIT - SMEM_ALIGN - BAR_BYTES - EPI_TOTAL) / per;
    return std::min(s, 12);
}

size_t smem_bytes(int bn, int stages) {
    return (size_t)SMEM_ALIGN + (size_t)stages * (A_BYTES + bn * 128) + EPI_TOTAL + BAR_BYTES;
}

template <int BN, bool FP8, int G, int FMODE = 0>
gbconv_status_t launch_kernel(const FwdParams<G> &prm, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fwd_kernel<BN, FP8, G, FMODE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    size_t smem = smem_bytes(BN, prm.stages);
    return cuda_status(launch_pdl(tc_fwd_kernel<BN, FP8, G, FMODE>, dim3(grid),
                                  dim3(EpiShape<BN>::threads), smem, st, prm));
}

template <int BN, int FMODE>
gbconv_status_t launch_single(const FwdParams<1> &prm, bool fp8, int grid, cudaStream_t st) {
    return fp8 ? launch_kernel<BN, true, 1, FMODE>(prm, grid, st)
               : launch_kernel<BN, false, 1, FMODE>(prm, grid, st);
}

// Fills pa, tmA, tmB for one problem; bn is the tile width used.
gbconv_status_t setup_problem(const Dims &d, int bn, const void *x, const void *w,
                              const float *bias, const float *x_scale, const float *w_scale,
                              void *y, ProbArgs &pa, CUtensorMap &ta, CUtensorMap &tb,
                              CUtensorMap &ty) {
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    const int eb = fp8 ? 1 : 2;
    const int ke = 128 / eb;
    const CUtensorMapDataType in_t =
        fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // A 1x1, stride-1, unpadded convolution reads x as the plain matrix [N*H*W][C].
    const bool a_tiled = d.R == 1 && d.S == 1 && d.u == 1 && d.v == 1 && d.ph == 0 && d.pw == 0;
    gbconv_status_t s;
    if (a_tiled) {
        uint64_t adims[2] = {(uint64_t)d.C, (uint64_t)d.M()};
        uint64_t astr[1] = {(uint64_t)d.xstride() * eb};
        uint32_t abox[2] = {(uint32_t)ke, (uint32_t)BM};
        s = encode_tiled(&ta, in_t, 2, x, adims, astr, abox, CU_TENSOR_MAP_SWIZZLE_128B);
    } else {
        s = encode_im2col_act(&ta, d, x, eb, ke, BM);
    }
    if (s != GBCONV_OK) return s;
    // y [M][K]: stored in 32-row x 32-column chunks (BF16: 64-byte rows, FP32: 128-byte rows)
    const bool of32 = d.out_dtype == GBCONV_F32;
    uint64_t ydims[2] = {(uint64_t)d.K, (uint64_t)d.M()};
    uint64_t ystr[1] = {(uint64_t)d.ystride() * (of32 ? 4 : 2)};
    uint32_t ybox[2] = {32, 32};
    s = encode_tiled(&ty, of32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     2, y, ydims, ystr, ybox,
                     of32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
    if (s != GBCONV_OK) return s;
    uint64_t dims[3] = {(uint64_t)d.C, (uint64_t)d.R * d.S, (uint64_t)d.K};
    uint64_t strides[2] = {(uint64_t)d.C * eb, (uint64_t)d.R * d.S * d.C * eb};
    uint32_t box[3] = {(uint32_t)ke, 1, (uint32_t)bn};
    s = encode_tiled(&tb, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     w, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    pa.M = (int)d.M();
    pa.P = d.P;
    pa.Q = d.Q;
    pa.pw = d.pw;
    pa.ph = d.ph;
    pa.u = d.u;
    pa.v = d.v;
    pa.dh = d.dh;
    pa.dw = d.dw;
    pa.S = d.S;
    pa.RS = d.R * d.S;
    pa.c_blocks = (d.C + ke - 1) / ke;
    pa.kb_per_tile = pa.RS * pa.c_blocks;
    pa.n_tiles = (d.K + bn - 1) / bn;
    pa.bn = bn;
    pa.K = d.K;
    pa.relu = (d.flags & GBCONV_FLAG_RELU) ? 1 : 0;
    pa.out_f32 = of32;
    pa.a_tiled = a_tiled;
    pa.bias = (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr;
    pa.x_scale = x_scale;
    pa.w_scale = w_scale;
    return GBCONV_OK;
}

int tiles_of(const ProbArgs &pa) { return ((pa.M + BM - 1) / BM) * pa.n_tiles; }

}  // namespace

bool tc_fwd_supported(const Dims &d) {
    if (d.layout != GBCONV_NHWC) return false;
    if (d.in_dtype == GBCONV_BF16) {
        if (d.out_dtype != GBCONV_BF16 && d.out_dtype != GBCONV_F32) return false;
        if (d.C % 8 || d.K % 8) return false;
    } else if (d.in_dtype == GBCONV_E4M3) {
        if (d.out_dtype != GBCONV_BF16) return false;
        if (d.C % 16 || d.K % 8) return false;
    } else {
        return false;
    }
    // im2col bounding-box corners are signed 8-bit for 4-D maps
    if (d.pw > 127 || d.ph > 127) return false;
    if (d.pw - d.dw * (d.S - 1) < -128 || d.ph - d.dh * (d.R - 1) < -128) return false;
    if (d.dw * (d.S - 1) > 65535 || d.dh * (d.R - 1) > 65535) return false;
    if (d.u > 8 || d.v > 8) return false;  // TMA traversal stride limit
    if (d.M() >= (1ll << 31)) return false;
    return true;
}

TcConfig tc_fwd_default_config(const Dims &d) {
    TcConfig c{};
    if (d.K <= 32)
        c.block_n = 32;
    else if (d.K <= 64)
        c.block_n = 64;
    else if (d.K <= 128 || d.K % 256 != 0)
        c.block_n = 128;
    else
        c.block_n = 256;
    c.stages = max_stages(c.block_n);
    c.split_k = 1;
    c.raster = 0;
    c.algo = GBCONV_ALGO_AUTO;
    return c;
}

gbconv_status_t launch_tc_fwd(const Dims &d, const TcConfig &cfg_in, const void *x,
                              const void *w, const float *bias, const float *x_scale,
                              const float *w_scale, void *y, cudaStream_t st, const Fused &fz) {
    TcConfig cfg = cfg_in;
    if (cfg.block_n != 32 && cfg.block_n != 64 && cfg.block_n != 128 && cfg.block_n != 256)
        return GBCONV_ERR_INVALID_ARG;
    // Automatic choice: for layers with more than one filter tap, the
    // transposed band kernel when the output channels fit one 128-row MMA
    // (any stride up to 4, by phase decomposition), else the shifted-band
    // kernel for stride-1 layers whose filter fits in shared memory. A 1x1
    // layer gains nothing from a band and would compute the extended rows'
    // spare columns.
    // Above 128 output channels the band kernel takes the layer only when 256-wide
    // pixel-major tiles would be ragged (K not a multiple of 256) and the filter
    // cannot stay resident in the pixel-major band kernel (measured: K = 192 is
    // 30 % faster on the band kernel, K = 256 20-35 % slower).
    // The pixel-major band kernel (output pixels on M, filter resident, one SM
    // or a pair of SMs per MMA) runs when the config asks for it (multi-tap
    // BF16 layers with up to 128 output channels, no fused scale or residual).
    // The automatic choice does not take it: on the ResNet 3x3 layers it
    // measured slower than the transposed band kernel (L2 17.4 against 15.0
    // us, the strided L4 20.2 against 14.0 us).
    if (cfg.algo == GBCONV_ALGO_PBAND || cfg.algo == GBCONV_ALGO_PBAND_PAIR) {
        const int want = cfg.algo == GBCONV_ALGO_PBAND ? 1 : 2;
        const int form = (fz.alpha || fz.z) ? 0 : tc_fwd_p_form(d, want);
        if (form) return launch_tc_fwd_p(d, form, x, w, bias, y, st);
        return GBCONV_ERR_UNSUPPORTED;
    }
    if (cfg.algo == GBCONV_ALGO_SHIFT_T ||
        (cfg.algo == GBCONV_ALGO_AUTO && d.R * d.S > 1 &&
         (d.K <= 128 || (d.K % 256 != 0 && !tc_fwd_shift_preferred(d, cfg.block_n))))) {
        if (tc_fwd_t_tile(d))
            return launch_tc_fwd_t(d, x, w, bias, x_scale, w_scale, y, st, fz);
        if (cfg.algo == GBCONV_ALGO_SHIFT_T) return GBCONV_ERR_UNSUPPORTED;
    }
    if (cfg.algo == GBCONV_ALGO_SHIFT && tc_fwd_shift_supported(d, cfg.block_n))
        return launch_tc_fwd_shift(d, cfg, x, w, bias, x_scale, w_scale, y, st, fz);
    if (cfg.algo == GBCONV_ALGO_AUTO && d.R * d.S > 1 && tc_fwd_shift_preferred(d, cfg.block_n))
        return launch_tc_fwd_shift(d, cfg, x, w, bias, x_scale, w_scale, y, st, fz);
    if (cfg.algo == GBCONV_ALGO_SHIFT) return GBCONV_ERR_UNSUPPORTED;  // not a stride-1 band layer
    if (cfg.stages < 2 || cfg.stages > max_stages(cfg.block_n)) cfg.stages = max_stages(cfg.block_n);
    if (d.M() == 0) return GBCONV_OK;
    FwdParams<1> prm;
    memset(&prm, 0, sizeof(prm));
    gbconv_status_t s = setup_problem(d, cfg.block_n, x, w, bias, x_scale, w_scale, y, prm.pa[0],
                                      prm.tmA[0], prm.tmB[0], prm.tmY[0]);
    if (s != GBCONV_OK) return s;
    prm.count = 1;
    prm.tile_start[0] = 0;
    prm.num_tiles = tiles_of(prm.pa[0]);
    prm.tile_start[1] = prm.num_tiles;
    prm.stages = cfg.stages;
    prm.raster = cfg.raster;
    prm.alpha = fz.alpha;
    prm.z = fz.z;
    if (fz.z && d.out_dtype == GBCONV_BF16) {  // residual tiles by TMA, y's store map shape
        uint64_t zd[2] = {(uint64_t)d.K, (uint64_t)d.M()};
        uint64_t zs[1] = {(uint64_t)d.ystride() * 2};
        uint32_t zb[2] = {32, 32};
        s = encode_tiled(&prm.tmZ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, fz.z, zd, zs, zb,
                         CU_TENSOR_MAP_SWIZZLE_64B);
        if (s != GBCONV_OK) return s;
        prm.z_tma = 1;
    }
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    int grid = std::min(prm.num_tiles, sm_count());
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    if (prm.z_tma) {
        switch (cfg.block_n) {
            case 32: return launch_single<32, 2>(prm, fp8, grid, st);
            case 64: return launch_single<64, 2>(prm, fp8, grid, st);
            case 128: return launch_single<128, 2>(prm, fp8, grid, st);
            default: return launch_single<256, 2>(prm, fp8, grid, st);
        }
    }
    if (fz.alpha || fz.z) {
        switch (cfg.block_n) {
            case 32: return launch_single<32, 1>(prm, fp8, grid, st);
            case 64: return launch_single<64, 1>(prm, fp8, grid, st);
            case 128: return launch_single<128, 1>(prm, fp8, grid, st);
            default: return launch_single<256, 1>(prm, fp8, grid, st);
        }
    }
    switch (cfg.block_n) {
        case 32: return launch_single<32, 0>(prm, fp8, grid, st);
        case 64: return launch_single<64, 0>(prm, fp8, grid, st);
        case 128: return launch_single<128, 0>(prm, fp8, grid, st);
        default: return launch_single<256, 0>(prm, fp8, grid, st);
    }
}

// Grouped: problems are ordered by descending per-tile work (filter taps x
// channel blocks x tile width) so that the static round-robin tile walk hands
// every CTA a similar mix of long and short tiles.
gbconv_status_t launch_tc_grouped(int count, const Dims *d, const TcConfig *cfg,
                                  const void *const *x, const void *const *w,
                                  const float *const *bias, void *const *y, cudaStream_t st) {
    for (int base = 0; base < count; base += GMAX) {
        const int cnt = std::min(GMAX, count - base);
        std::vector<int> order(cnt);
        for (int i = 0; i < cnt; ++i) order[i] = base + i;
        auto work = [&](int i) {
            const int ke = 64;
            long long kb = (long long)d[i].R * d[i].S * ((d[i].C + ke - 1) / ke);
            return kb * cfg[i].block_n;
        };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
        static FwdParams<GMAX> prm;  // large: keep off the stack
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        memset(&prm, 0, sizeof(prm));
        int tiles = 0, slot = 0;
        for (int oi = 0; oi < cnt; ++oi) {
            const int i = order[oi];
            if (d[i].M() == 0) continue;
            if (cfg[i].block_n != 32 && cfg[i].block_n != 64 && cfg[i].block_n != 128 &&
                cfg[i].block_n != 256)
                return GBCONV_ERR_INVALID_ARG;
            gbconv_status_t s = setup_problem(d[i], cfg[i].block_n, x[i], w[i], bias[i], nullptr,
                                              nullptr, y[i], prm.pa[slot], prm.tmA[slot],
                                              prm.tmB[slot], prm.tmY[slot]);
            if (s != GBCONV_OK) return s;
            prm.tile_start[slot] = tiles;
            tiles += tiles_of(prm.pa[slot]);
            ++slot;
        }
        if (slot == 0) continue;
        prm.tile_start[slot] = tiles;
        prm.count = slot;
        prm.num_tiles = tiles;
        prm.stages = max_stages(256);
        prm.raster = 0;
        prm.guard = make_guard();
        if (!prm.guard.err) return GBCONV_ERR_CUDA;
        int grid = std::min(tiles, sm_count());
        gbconv_status_t s = launch_kernel<256, false, GMAX>(prm, grid, st);
        if (s != GBCONV_OK) return s;
    }
    return GBCONV_OK;
}

}  // namespace gbc
