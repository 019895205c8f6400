// tc_fwd_p.cu -- pixel-major band kernel for multi-tap layers with at most 128
// output channels, on one SM or on a pair of SMs (tcgen05 cta_group::2).
//
// The forward pass of a convolutional layer (paper Sec. 5.B) as the implicit
// GEMM D[e][k] = sum_{(r,s), c} band[e + shift(r,s)][c] * W[k][(r,s)][c], with
// the output positions e on the MMA's M (128 rows per SM) and the output
// channels on N:
//
//  * Strides by phase decomposition (as in tc_fwd_t.cu): tap (r, s) of output
//    (p, q) reads input row u*(p + i) + a - ph with a = (r*dh) mod u,
//    i = (r*dh) div u (columns likewise with v, b, j), so within a phase
//    (a, b) every tap is the shift (i, j) of one phase image. One TMA box with
//    element strides (v, u) loads a band of a phase image; stride 1 is the
//    single phase.
//  * Output positions are indexed on extended rows of Wx = Q + max j columns
//    (no power-of-two rounding): e = row * Wx + q. A tile is TR whole output
//    rows of one image, TR * Wx <= 128 positions; positions past TR * Wx and
//    columns q >= Q are computed and discarded.
//  * A operand: 128 band rows starting at the tap's shift i*Wx + j (any
//    128-byte row of a swizzled buffer is a valid start; measured on GB300 at
//    the full MMA rate). B operand: the filter tile (tap, 64-channel block),
//    resident in shared memory for the whole kernel, loaded once in MMA order
//    with a barrier per group of tiles so the first MMAs wait only for the
//    first tiles.
//  * Pair mode (cta_group::2): the two SMs of a cluster compute one 256-row
//    MMA each time, each on its own tile's band (its 128 rows of M) while each
//    holds half of the filter's output channels (its half of N). One thread of
//    the even CTA issues every MMA. Each CTA's band and filter loads count on
//    the even CTA's barriers; the MMA commits arrive on both CTAs' barriers;
//    the odd CTA's epilogue releases the accumulator on the even CTA's barrier.
//    With 128 output channels this keeps the filter resident (half of it per
//    SM), where a single SM would have to stream it per tile.
//  * TMEM: 256 columns = 256 / BN accumulators used in turn, so the epilogue
//    of a tile overlaps the MMAs of the next ones.
//  * Epilogue: 8 warps, two per TMEM lane quarter; a thread owns one output
//    position (its TMEM lane) and 32 consecutive channels per 32x32b load:
//    bias, ReLU, round to BF16 (or keep FP32) and 16-byte stores straight to
//    y, whose channels are contiguous (NHWC). No shared-memory staging, so the
//    band ring can take most of shared memory.
//
// Warp roles: warp 0 loads the bands (one thread), warp 1 issues the MMAs
// (one thread; in pair mode only the even CTA's), warps 2-9 the epilogue,
// warp 10 loads the filter (one tile per lane). Every wait on an mbarrier is
// bounded; on a timeout the kernel records DEVERR_TIMEOUT, stops its loops
// (in pair mode both CTAs') and leaves through the common exit, which frees
// TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int PM = 128;                         // output positions per CTA tile
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quarter
constexpr int FILTER_WARP = 2 + EPI_WARPS;
constexpr int NTHREADS = 32 * (3 + EPI_WARPS);  // band producer, MMA, epilogue, filter producer
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 2048;  // barriers, then the per-tap descriptor offsets
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_SA = 6;                       // band ring stages
constexpr int MAX_WG = 32;                      // barriers over the resident filter
constexpr int MAX_NACC = 4;
constexpr int MAX_STRIDE = 4;
constexpr int MAX_PHASES = MAX_STRIDE * MAX_STRIDE;
constexpr int MAX_TAPS = 64;
constexpr int TCOLS = 256;                      // TMEM columns allocated
constexpr int KE = 64;                          // BF16 channels per 128-byte row

struct PParams {
    CUtensorMap tmX;  // x [N][H][W][C], box {64, v*Wx, u*nr, 1}, element strides {1, v, u, 1}
    CUtensorMap tmW;  // w [K][R*S][C], box {64, 1, filter rows of one CTA}
    int P, Q, K;
    int u;
    int Wx, TR, n_pos;  // n_pos = TR * Wx <= 128
    int c_blocks, n_taps;
    // phase f: band origin (column b - pw, row offset a - ph), taps [end[f-1], end[f])
    int n_phase;
    int ph_w0[MAX_PHASES], ph_h0[MAX_PHASES], ph_end[MAX_PHASES];
    uint16_t tap_t[MAX_TAPS];      // filter tap r*S + s
    uint16_t tap_shift[MAX_TAPS];  // band row offset i*Wx + j
    int p_tiles, num_tiles, num_units;  // a unit is one tile (one SM) or two (a pair)
    int band_bytes, band_stride, stages;
    int w_tiles, wper;  // resident filter tiles (channel block, then tap table), tiles per barrier
    int relu, out_f32;
    const float *bias;
    void *y;  // [N][P][Q][K], BF16 or FP32
    Guard guard;
};

static_assert(sizeof(PParams) <= 4096, "pixel-major band kernel parameters too large");

struct PTile {
    int n, p0;
    bool valid;
};

// CTA tile of a unit: a pair's odd CTA past the last tile recomputes the last
// tile (its loads keep the pair's byte counts) and stores nothing.
template <bool PAIR>
__device__ __forceinline__ PTile ptile(const PParams &p, int unit, uint32_t rank) {
    int t = PAIR ? 2 * unit + (int)rank : unit;
    PTile r;
    r.valid = t < p.num_tiles;
    if (!r.valid) t = p.num_tiles - 1;
    r.n = t / p.p_tiles;
    r.p0 = (t - r.n * p.p_tiles) * p.TR;
    return r;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a -> low half
    return *reinterpret_cast<uint32_t *>(&h);
}

// The MMAs of one band: NT taps x 4 K-steps of 16 channels, straight-line
// code with the taps' descriptor offsets in registers. The issuing thread must
// keep up with MMAs of 25-35 ns, and the tensor core's queue of MMA
// instructions is short: any latency between two MMAs (a loop, a table lookup,
// a division) leaves the tensor core idle.
template <int NT, bool PAIR>
__device__ __forceinline__ void issue_taps(uint32_t d, uint64_t a0, uint64_t b0, const uint32_t *aoff,
                                           const uint32_t *boff, uint32_t idesc, uint32_t &accum) {
    uint32_t ao[NT], bo[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        ao[t] = aoff[t];
        bo[t] = boff[t];
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t ad = a0 + ao[t] + 2 * k, bd = b0 + bo[t] + 2 * k;
            if (PAIR)
                ptx::mma_f16_pair(d, ad, bd, idesc, accum);
            else
                ptx::mma_f16(d, ad, bd, idesc, accum);
            accum = 1;
        }
}

template <bool PAIR>
__device__ __forceinline__ void issue_band(int nt, uint32_t d, uint64_t a0, uint64_t b0,
                                           const uint32_t *aoff, const uint32_t *boff, uint32_t idesc,
                                           uint32_t &accum) {
    switch (nt) {
        case 1: issue_taps<1, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        case 2: issue_taps<2, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        case 3: issue_taps<3, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        case 4: issue_taps<4, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        case 6: issue_taps<6, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        case 9: issue_taps<9, PAIR>(d, a0, b0, aoff, boff, idesc, accum); return;
        default:
            for (int t0 = 0; t0 < nt; t0 += 4) {  // other tap counts in runs of up to four
                const int n = nt - t0 < 4 ? nt - t0 : 4;
                if (n == 4)
                    issue_taps<4, PAIR>(d, a0, b0, aoff + t0, boff + t0, idesc, accum);
                else if (n == 3)
                    issue_taps<3, PAIR>(d, a0, b0, aoff + t0, boff + t0, idesc, accum);
                else if (n == 2)
                    issue_taps<2, PAIR>(d, a0, b0, aoff + t0, boff + t0, idesc, accum);
                else
                    issue_taps<1, PAIR>(d, a0, b0, aoff + t0, boff + t0, idesc, accum);
            }
    }
}

template <int BN, bool PAIR>
__global__ void __launch_bounds__(NTHREADS, 1) tc_fwd_p_kernel(const __grid_constant__ PParams prm) {
    constexpr int NACC = TCOLS / BN;          // accumulators (4 for 64 channels, 2 for 128)
    constexpr int BNH = PAIR ? BN / 2 : BN;   // filter rows (output channels) held by this CTA
    constexpr int W_TILE = BNH * 128;         // one filter tile (tap, channel block)
    constexpr int NCH = BN / 32;              // 32-column chunks of an accumulator
    static_assert(NACC <= MAX_NACC, "too many accumulators");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int SA = prm.stages;
    uint8_t *sA = base;                          // band ring
    uint8_t *sW = sA + SA * prm.band_stride;     // resident filter
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + prm.w_tiles * W_TILE);
    uint64_t *fullA = bars;                      // [MAX_SA]
    uint64_t *emptyA = fullA + MAX_SA;           // [MAX_SA]
    uint64_t *tfull = emptyA + MAX_SA;           // [MAX_NACC]
    uint64_t *tempty = tfull + MAX_NACC;         // [MAX_NACC]
    uint64_t *wres = tempty + MAX_NACC;          // [MAX_WG]
    uint64_t *done = wres + MAX_WG;              // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    // per-tap descriptor offsets (16-byte units): band row shift, filter tile
    uint32_t *s_aoff = reinterpret_cast<uint32_t *>(bars) + 128;  // [MAX_TAPS]
    uint32_t *s_boff = s_aoff + MAX_TAPS;                         // [MAX_TAPS]
    int *s_tap0 = reinterpret_cast<int *>(s_boff + MAX_TAPS);     // [MAX_PHASES + 1]: phase f's taps

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? ptx::cluster_rank() : 0u;
    const bool leader = rank == 0;
    const uint64_t lim = prm.guard.wait_ns;
    const int unit0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int ustep = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int n_wgrp = (prm.w_tiles + prm.wper - 1) / prm.wper;

    if (threadIdx.x == 0) {
        for (int i = 0; i < SA; ++i) {
            ptx::mbar_init(&fullA[i], 1);
            ptx::mbar_init(&emptyA[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            ptx::mbar_init(&tfull[i], 1);
            ptx::mbar_init(&tempty[i], (PAIR ? 2 : 1) * EPI_WARPS);
        }
        for (int g = 0; g < n_wgrp; ++g) ptx::mbar_init(&wres[g], 1);
        ptx::mbar_init(done, 1);
        for (int i = 0; i < prm.n_taps; ++i) {
            s_aoff[i] = (uint32_t)prm.tap_shift[i] << 3;  // 128-byte rows = 8 units
            s_boff[i] = (uint32_t)i * (W_TILE >> 4);
        }
        s_tap0[0] = 0;
        for (int f = 0; f < prm.n_phase; ++f) s_tap0[f + 1] = prm.ph_end[f];
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        if (PAIR) {
            ptx::tmem_alloc_pair(tmem_slot, TCOLS);
            ptx::tmem_relinquish_pair();
        } else {
            ptx::tmem_alloc(tmem_slot, TCOLS);
            ptx::tmem_relinquish();
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (PAIR) ptx::cluster_sync();  // the peer's barriers exist before any remote arrive
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the even CTA's barriers as cluster addresses (pair mode)
    const uint32_t fullA_l = PAIR ? ptx::cluster_addr(ptx::smem_addr(fullA), 0) : 0u;
    const uint32_t tempty_l = PAIR ? ptx::cluster_addr(ptx::smem_addr(tempty), 0) : 0u;
    const uint32_t wres_l = PAIR ? ptx::cluster_addr(ptx::smem_addr(wres), 0) : 0u;
    const uint32_t abort_peer =
        PAIR ? ptx::cluster_addr(ptx::smem_addr(const_cast<int *>(abort_flag)), rank ^ 1u) : 0u;

    // Descriptors and first inputs do not depend on earlier kernels: the first
    // tile's bands (warp 0, a band per lane) and this CTA's filter tiles (the
    // filter warp, a tile per lane) go into L2 while the previous kernel drains
    // (L2 stays coherent with its writes; the loads into shared memory come
    // after the dependency wait). A prefetch holds its issuing thread for about
    // as long as a load, so the lanes share them.
    if ((warp == 0 || warp == FILTER_WARP) && unit0 < prm.num_units) {
        if (lane == 0) ptx::prefetch_tmap(warp == 0 ? &prm.tmX : &prm.tmW);
        __syncwarp();
        if (warp == 0) {
            const PTile T = ptile<PAIR>(prm, unit0, rank);
            for (int i = lane; i < prm.c_blocks * prm.n_phase; i += 32) {
                const int cb = i / prm.n_phase, f = i - cb * prm.n_phase;
                ptx::tma_prefetch_4d(&prm.tmX, cb * KE, prm.ph_w0[f], prm.u * T.p0 + prm.ph_h0[f], T.n);
            }
        } else {
            for (int seq = lane; seq < prm.w_tiles; seq += 32) {
                const int cb = seq / prm.n_taps;
                ptx::tma_prefetch_3d(&prm.tmW, cb * KE, prm.tap_t[seq - cb * prm.n_taps],
                                     (int)rank * BNH);
            }
        }
    }
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();

    // Bounded wait; in a pair with cluster-scope acquire (the barriers there
    // also receive the other CTA's arrivals).
    auto wait = [&](uint64_t *bar, uint32_t parity, const volatile int *ab) {
        return PAIR ? ptx::mbar_wait_cluster(bar, parity, lim, ab) : ptx::mbar_wait(bar, parity, lim, ab);
    };
    // Record a failed wait: stop this CTA's loops and, in a pair, the peer's.
    auto fail = [&]() {
        *abort_flag = 1;
        if (PAIR) asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(abort_peer), "r"(1) : "memory");
        atomicOr(prm.guard.err, DEVERR_TIMEOUT);
    };
    const bool skip = prm.guard.skip_loads != 0;

    if (warp == 0) {
        // ------------------------------ band producer ------------------------------
        if (lane == 0) {
            int sa = 0, issued = 0;
            uint32_t pa = 0;
            bool ok = true;
            for (int unit = unit0; ok && unit < prm.num_units; unit += ustep) {
                const PTile T = ptile<PAIR>(prm, unit, rank);
                for (int cb = 0; ok && cb < prm.c_blocks; ++cb)
                    for (int f = 0; f < prm.n_phase; ++f) {
                        if (!wait(&emptyA[sa], pa ^ 1, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        if (!skip) {
                            uint8_t *dst = sA + sa * prm.band_stride;
                            const int h0 = prm.u * T.p0 + prm.ph_h0[f];
                            if (PAIR) {
                                if (leader)
                                    ptx::mbar_arrive_expect_tx(&fullA[sa], 2u * (uint32_t)prm.band_bytes);
                                ptx::tma_load_4d_pair(dst, &prm.tmX, fullA_l + 8u * sa, cb * KE,
                                                      prm.ph_w0[f], h0, T.n);
                            } else {
                                ptx::mbar_arrive_expect_tx(&fullA[sa], (uint32_t)prm.band_bytes);
                                ptx::tma_load_4d(dst, &prm.tmX, &fullA[sa], cb * KE, prm.ph_w0[f], h0, T.n);
                            }
                            ++issued;
                        }
                        if (++sa == SA) {
                            sa = 0;
                            pa ^= 1;
                        }
                    }
            }
            // Drain: every stage this producer filled has been consumed by the
            // MMAs (so its load landed and, in a pair, the commits releasing it
            // reached this CTA) before shared memory is given back.
            int st = sa;
            uint32_t ph = pa;
            for (int i = 0; i < min(issued, SA); ++i) {
                if (st == 0) {
                    st = SA;
                    ph ^= 1;
                }
                --st;
                if (!wait(&emptyA[st], ph, abort_flag)) fail();
            }
        }
    } else if (warp == FILTER_WARP) {
        // ----------------------------- filter producer -----------------------------
        // Every tile of this CTA's filter rows once, in MMA order, one per lane;
        // each group's byte count is announced (by the even CTA, for both CTAs of
        // a pair) before any of its loads.
        for (int s0 = 0; !skip && s0 < prm.w_tiles; s0 += 32) {
            const int seq = s0 + lane;
            const bool act = seq < prm.w_tiles;
            if (act && seq % prm.wper == 0 && leader) {
                const int g = seq / prm.wper;
                const uint32_t bytes = (uint32_t)(min(prm.wper, prm.w_tiles - g * prm.wper) * W_TILE);
                ptx::mbar_arrive_expect_tx(&wres[g], PAIR ? 2u * bytes : bytes);
            }
            __syncwarp();
            if (act) {
                const int cb = seq / prm.n_taps;
                const int t = prm.tap_t[seq - cb * prm.n_taps];
                if (PAIR)
                    ptx::tma_load_3d_pair(sW + seq * W_TILE, &prm.tmW, wres_l + 8u * (seq / prm.wper),
                                          cb * KE, t, (int)rank * BNH);
                else
                    ptx::tma_load_3d(sW + seq * W_TILE, &prm.tmW, &wres[seq / prm.wper], cb * KE, t, 0);
            }
            __syncwarp();
        }
        // The filter loads have landed before the CTA leaves: the even CTA waits
        // for every group (in a pair they also count the odd CTA's loads, and the
        // odd CTA leaves only after the even one, at the final cluster barrier).
        if (lane == 0 && !skip && leader) {
            volatile int zero = 0;
            for (int g = 0; g < n_wgrp; ++g)
                if (!wait(&wres[g], 0, &zero)) fail();
        }
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ----------------------------
        if (lane == 0 && leader) {
            bool ok = true;
            uint32_t idesc = ptx::idesc_bf16(BN);
            idesc = (idesc & ~(0x1Fu << 24)) | ((uint32_t)((PAIR ? 256 : 128) >> 4) << 24);
            const uint64_t wdb = ptx::sdesc_kmajor_sw128(ptx::smem_addr(sW));
            const uint64_t adb0 = ptx::sdesc_kmajor_sw128(ptx::smem_addr(sA));
            const uint32_t a_stage = (uint32_t)prm.band_stride >> 4;        // descriptor units per stage
            const uint32_t b_cblock = (uint32_t)prm.n_taps * (W_TILE >> 4);  // per channel block
            const int c_blocks = prm.c_blocks, n_phase = prm.n_phase;
            // the barriers this thread commits to, as cluster addresses (pair mode)
            const uint32_t empty_own = ptx::smem_addr(emptyA), tfull_own = ptx::smem_addr(tfull);
            const uint32_t empty_peer = PAIR ? ptx::cluster_addr(empty_own, 1) : 0u;
            const uint32_t tfull_peer = PAIR ? ptx::cluster_addr(tfull_own, 1) : 0u;
            int sa = 0, local = 0;
            uint32_t pa = 0;
            for (int unit = unit0; ok && unit < prm.num_units; unit += ustep, ++local) {
                const int acc = local % NACC;
                const uint32_t aph = (uint32_t)(local / NACC) & 1u;
                if (!wait(&tempty[acc], aph ^ 1, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                uint32_t accum = 0;
                for (int cb = 0; ok && cb < c_blocks; ++cb) {
                    for (int f = 0; f < n_phase; ++f) {
                        const int t0 = s_tap0[f], t1 = s_tap0[f + 1];
                        if (local == 0) {
                            // the first tile waits for the filter groups of each band
                            // as it reaches them (later tiles find them all resident)
                            const int g0 = (cb * prm.n_taps + t0) / prm.wper;
                            const int g1 = (cb * prm.n_taps + t1 - 1) / prm.wper;
                            for (int g = g0; ok && g <= g1; ++g)
                                if (!wait(&wres[g], 0, abort_flag)) {
                                    fail();
                                    ok = false;
                                }
                            if (!ok) break;
                        }
                        if (!wait(&fullA[sa], pa, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        // descriptors by addition (the start-address field cannot carry:
                        // shared addresses stay below 256 KB)
                        issue_band<PAIR>(t1 - t0, d, adb0 + (uint64_t)(sa * a_stage),
                                         wdb + (uint64_t)(cb * b_cblock), s_aoff + t0, s_boff + t0, idesc,
                                         accum);
                        if (PAIR) {
                            ptx::mma_commit_pair(empty_own + 8u * sa);
                            ptx::mma_commit_pair(empty_peer + 8u * sa);
                        } else {
                            ptx::mma_commit(&emptyA[sa]);
                        }
                        if (++sa == SA) {
                            sa = 0;
                            pa ^= 1;
                        }
                    }
                }
                if (!ok) break;
                if (PAIR) {
                    ptx::mma_commit_pair(tfull_own + 8u * acc);
                    ptx::mma_commit_pair(tfull_peer + 8u * acc);
                } else {
                    ptx::mma_commit(&tfull[acc]);
                }
            }
            if (PAIR)
                ptx::mma_commit_pair(ptx::smem_addr(done));
            else
                ptx::mma_commit(done);
            volatile int zero = 0;
            if (!wait(done, 0, &zero)) fail();
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int ew = warp - 2;       // 0..7
        const int quarter = warp & 3;  // TMEM lane quarter this warp may read
        const int half = ew >> 2;      // chunks j = half, half + 2, ...
        const int e = quarter * 32 + lane;  // this thread's position in the tile
        const int erow = e / prm.Wx, ecol = e - erow * prm.Wx;
        int local = 0;
        for (int unit = unit0; unit < prm.num_units; unit += ustep, ++local) {
            const PTile T = ptile<PAIR>(prm, unit, rank);
            const int acc = local % NACC;
            const uint32_t aph = (uint32_t)(local / NACC) & 1u;
            const int p = T.p0 + erow;
            const bool valid = T.valid && e < prm.n_pos && p < prm.P && ecol < prm.Q;
            const size_t yrow = ((size_t)T.n * prm.P + (size_t)p) * prm.Q + (size_t)ecol;
            if (!wait(&tfull[acc], aph, abort_flag)) {
                fail();
                break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int j = half; j < NCH; j += 2) {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(acc * BN + j * 32),
                                        v);
                ptx::tmem_ld_wait();
                ptx::reg_fence(v);
                if (j + 2 >= NCH) {  // this warp's last read of the accumulator
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (PAIR)
                            ptx::mbar_arrive_cluster(tempty_l + 8u * acc);
                        else
                            ptx::mbar_arrive(&tempty[acc]);
                    }
                }
                const int k0 = j * 32;
                if (!valid || k0 >= prm.K) continue;
                float a[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    float t = __uint_as_float(v[i]);
                    if (prm.bias && k0 + i < prm.K) t += __ldg(prm.bias + k0 + i);
                    if (prm.relu) t = fmaxf(t, 0.f);
                    a[i] = t;
                }
                if (prm.out_f32) {
                    float *yp = static_cast<float *>(prm.y) + yrow * prm.K + k0;
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (k0 + 4 * c < prm.K)
                            *reinterpret_cast<float4 *>(yp + 4 * c) =
                                make_float4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
                } else {
                    __nv_bfloat16 *yp = static_cast<__nv_bfloat16 *>(prm.y) + yrow * prm.K + k0;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (k0 + 8 * c < prm.K)
                            *reinterpret_cast<uint4 *>(yp + 8 * c) =
                                make_uint4(pack2(a[8 * c], a[8 * c + 1]), pack2(a[8 * c + 2], a[8 * c + 3]),
                                           pack2(a[8 * c + 4], a[8 * c + 5]), pack2(a[8 * c + 6], a[8 * c + 7]));
                }
            }
        }
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    if (PAIR) ptx::cluster_sync();  // neither CTA leaves while the other may still signal it
    ptx::tc_fence_after();
    if (warp == 1) {
        if (PAIR)
            ptx::tmem_dealloc_pair(tmem_base, TCOLS);
        else
            ptx::tmem_dealloc(tmem_base, TCOLS);
    }
}

// ---------------------------------------------------------------------------
// host side

struct PPlan {
    int bn;
    bool pair;
    int Wx, TR, nr, p_tiles;
    int band_bytes, band_stride, stages;
    int c_blocks, w_tiles, wper;
    long long num_tiles;
};

int phase_of(const Dims &d, int r, int s) { return ((r * d.dh) % d.u) * d.v + (s * d.dw) % d.v; }

bool make_pplan(const Dims &d, bool pair, PPlan *pl) {
    if (!tc_fwd_supported(d) || d.in_dtype != GBCONV_BF16) return false;
    if (d.R * d.S < 2 || d.R * d.S > MAX_TAPS) return false;
    if (d.u > MAX_STRIDE || d.v > MAX_STRIDE) return false;
    if (d.K > 128) return false;
    PPlan p{};
    p.bn = d.K <= 64 ? 64 : 128;
    p.pair = pair;
    const int imax = ((d.R - 1) * d.dh) / d.u, jmax = ((d.S - 1) * d.dw) / d.v;
    p.Wx = d.Q + jmax;
    if (p.Wx > PM || p.Wx * d.v > 256) return false;
    const int tr_max = std::min(PM / p.Wx, d.P);
    p.p_tiles = (d.P + tr_max - 1) / tr_max;
    p.TR = (d.P + p.p_tiles - 1) / p.p_tiles;  // rows spread evenly over the tiles
    p.nr = p.TR + imax;
    if (p.nr * d.u > 256) return false;
    p.band_bytes = 128 * p.Wx * p.nr;
    const int max_shift = imax * p.Wx + jmax;
    const int rows = std::max(p.Wx * p.nr, PM + max_shift);  // garbage rows stay inside the stage
    p.band_stride = (rows * 128 + 1023) / 1024 * 1024;
    p.c_blocks = (d.C + KE - 1) / KE;
    p.w_tiles = d.R * d.S * p.c_blocks;
    const int w_tile = (pair ? p.bn / 2 : p.bn) * 128;
    const long long budget = (long long)SMEM_LIMIT - SMEM_ALIGN - BAR_BYTES - (long long)p.w_tiles * w_tile;
    if (budget < 2ll * p.band_stride) return false;
    p.stages = (int)std::min<long long>(MAX_SA, budget / p.band_stride);
    p.wper = (p.w_tiles + MAX_WG - 1) / MAX_WG;
    p.num_tiles = (long long)d.N * p.p_tiles;
    if (p.num_tiles >= (1ll << 30) || d.M() >= (1ll << 31)) return false;
    *pl = p;
    return true;
}

// Tap table: taps grouped by phase (a, b), phases in order a*v + b, phases
// without taps left out.
void build_ptaps(const Dims &d, int Wx, PParams *prm) {
    int n = 0, f_out = 0;
    for (int a = 0; a < d.u; ++a)
        for (int b = 0; b < d.v; ++b) {
            const int start = n;
            for (int r = 0; r < d.R; ++r)
                for (int s = 0; s < d.S; ++s) {
                    if (phase_of(d, r, s) != a * d.v + b) continue;
                    const int i = (r * d.dh) / d.u, j = (s * d.dw) / d.v;
                    prm->tap_t[n] = (uint16_t)(r * d.S + s);
                    prm->tap_shift[n] = (uint16_t)(i * Wx + j);
                    ++n;
                }
            if (n == start) continue;
            prm->ph_w0[f_out] = b - d.pw;
            prm->ph_h0[f_out] = a - d.ph;
            prm->ph_end[f_out] = n;
            ++f_out;
        }
    prm->n_phase = f_out;
    prm->n_taps = n;
}

// Resident CTA pairs of the pair kernel (0 if the device cannot run them).
template <int BN>
int max_pairs() {
    static std::once_flag once;
    static int n = 0;
    std::call_once(once, [] {
        if (cudaFuncSetAttribute(tc_fwd_p_kernel<BN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMEM_LIMIT) != cudaSuccess)
            return;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * sm_count());
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = SMEM_LIMIT;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, tc_fwd_p_kernel<BN, true>, &cfg) == cudaSuccess) n = c;
    });
    return n;
}

template <int BN, bool PAIR>
gbconv_status_t launch_p(const PParams &prm, size_t smem, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fwd_p_kernel<BN, PAIR>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    int grid;
    if (PAIR) {
        const int pairs = max_pairs<BN>();
        if (pairs < 1) return GBCONV_ERR_UNSUPPORTED;
        grid = 2 * std::min(prm.num_units, pairs);
    } else {
        grid = std::min(prm.num_units, sm_count());
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 2 : 1;
    return cuda_status(cudaLaunchKernelEx(&cfg, tc_fwd_p_kernel<BN, PAIR>, prm));
}

}  // namespace

// 0: the kernel cannot take this layer; 1: one SM per tile; 2: a pair of SMs.
// want = 1 or 2 asks for that form, 0 for the automatic choice: one SM when
// its filter stays resident beside at least three band stages, else a pair.
int tc_fwd_p_form(const Dims &d, int want) {
    PPlan p;
    if (want == 1) return make_pplan(d, false, &p) ? 1 : 0;
    if (want == 2) return make_pplan(d, true, &p) ? 2 : 0;
    if (make_pplan(d, false, &p) && p.stages >= 3) return 1;
    if (make_pplan(d, true, &p)) return 2;
    return make_pplan(d, false, &p) ? 1 : 0;
}

gbconv_status_t launch_tc_fwd_p(const Dims &d, int form, const void *x, const void *w,
                                const float *bias, void *y, cudaStream_t st) {
    PPlan pl;
    if ((form != 1 && form != 2) || !make_pplan(d, form == 2, &pl)) return GBCONV_ERR_UNSUPPORTED;
    if (d.M() == 0) return GBCONV_OK;
    if (reinterpret_cast<uintptr_t>(y) % 16) return GBCONV_ERR_ALIGNMENT;  // 16-byte stores
    PParams prm;
    memset(&prm, 0, sizeof(prm));
    const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    uint64_t xd[4] = {(uint64_t)d.C, (uint64_t)d.W, (uint64_t)d.H, (uint64_t)d.N};
    uint64_t xs[3] = {(uint64_t)d.C * 2, (uint64_t)d.W * d.C * 2, (uint64_t)d.H * d.W * d.C * 2};
    uint32_t xb[4] = {(uint32_t)KE, (uint32_t)(d.v * pl.Wx), (uint32_t)(d.u * pl.nr), 1};
    uint32_t xe[4] = {1, (uint32_t)d.v, (uint32_t)d.u, 1};
    gbconv_status_t s = encode_tiled(&prm.tmX, bf, 4, x, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_128B, xe);
    if (s != GBCONV_OK) return s;
    const int rows = pl.pair ? pl.bn / 2 : pl.bn;
    uint64_t wd[3] = {(uint64_t)d.C, (uint64_t)d.R * d.S, (uint64_t)d.K};
    uint64_t wstr[2] = {(uint64_t)d.C * 2, (uint64_t)d.R * d.S * d.C * 2};
    uint32_t wbx[3] = {(uint32_t)KE, 1, (uint32_t)rows};
    s = encode_tiled(&prm.tmW, bf, 3, w, wd, wstr, wbx, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    prm.P = d.P;
    prm.Q = d.Q;
    prm.K = d.K;
    prm.u = d.u;
    prm.Wx = pl.Wx;
    prm.TR = pl.TR;
    prm.n_pos = pl.TR * pl.Wx;
    prm.c_blocks = pl.c_blocks;
    build_ptaps(d, pl.Wx, &prm);
    prm.p_tiles = pl.p_tiles;
    prm.num_tiles = (int)pl.num_tiles;
    prm.num_units = pl.pair ? (prm.num_tiles + 1) / 2 : prm.num_tiles;
    prm.band_bytes = pl.band_bytes;
    prm.band_stride = pl.band_stride;
    prm.stages = pl.stages;
    prm.w_tiles = pl.w_tiles;
    prm.wper = pl.wper;
    prm.relu = (d.flags & GBCONV_FLAG_RELU) ? 1 : 0;
    prm.out_f32 = d.out_dtype == GBCONV_F32;
    prm.bias = (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr;
    prm.y = y;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const size_t smem = (size_t)SMEM_ALIGN + (size_t)pl.stages * pl.band_stride +
                        (size_t)pl.w_tiles * rows * 128 + BAR_BYTES;
    if (smem > (size_t)SMEM_LIMIT) return GBCONV_ERR_UNSUPPORTED;
    if (pl.bn == 64) return pl.pair ? launch_p<64, true>(prm, smem, st) : launch_p<64, false>(prm, smem, st);
    return pl.pair ? launch_p<128, true>(prm, smem, st) : launch_p<128, false>(prm, smem, st);
}

}  // namespace gbc
