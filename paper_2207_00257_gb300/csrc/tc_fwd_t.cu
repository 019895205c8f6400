// tc_fwd_t.cu -- "transposed" shifted-band forward convolution for layers
// with at most 128 output channels and strides up to 4.
//
// Same idea as tc_fwd_shift.cu (one padded input band per channel block, every
// filter tap a row shift of it; forward pass of a convolutional layer, paper
// Sec. 5.B), but the GEMM is computed transposed:
//
//   D^T[k][e] = sum_{(r,s), c} W[k][(r,s)][c] * band[e + shift(r,s)][c]
//
// with M = KT output channels (64 or 128) and N = 256 extended output
// positions per tcgen05.mma. With pixels on M a 64-channel layer issues
// 128 x 64 x 16 MMAs, which sit on a ~27 ns per-instruction floor on GB300;
// with channels on M it issues half as many 64 x 256 x 16 MMAs (M = 64 runs
// at half the tensor rate), and a single thread issues every MMA of a CTA,
// so fewer, larger instructions win: 1.5x end to end on a 3x3 64->64 layer
// at 56x56, batch 32. With 128 channels the MMA is 128 x N at full rate.
//
//  * Strides by phase decomposition. Tap (r, s) of output (p, q) reads input
//    row u*p - ph + r*dh = u*(p + i) + a - ph with a = (r*dh) mod u,
//    i = (r*dh) div u, and likewise column v*(q + j) + b - pw. So the taps
//    split into u*v phases (a, b); within a phase every tap is the shift
//    (i, j) of one phase image X_ab[p'][q'] = x[u*p' + a - ph][v*q' + b - pw].
//    One band of a phase image is one TMA box with element strides (v, u)
//    over x. Stride 1 is the single phase (0, 0). A host-built table lists
//    the taps phase by phase (filter tap index, band row shift i*Wx + j);
//    phases without taps are skipped.
//  * Tile: TR output rows of one image as TR * Wx consecutive extended
//    positions (Wx = power of two >= Q + max j; TR <= 256 / Wx, chosen to
//    split the P rows into equal tiles), times KT output channels.
//  * A operand: filter tile W[(r,s), c block] = KT rows of 128 bytes, resident
//    in shared memory when the whole filter fits (loaded once, with barriers
//    per group of tiles so the first MMAs do not wait for the whole filter),
//    otherwise streamed in table order through its own ring, whose stages
//    hold up to four tiles each (one barrier wait and one commit per stage on
//    the MMA thread: each costs it about as much as an MMA's worth of time).
//  * B operand: 256 band rows starting at the tap's shift (K-major, 128-byte
//    swizzle; any 128-byte row is a valid start).
//  * TMEM: two 256-column accumulators. For M = 128 row k of D^T sits in lane
//    k; for M = 64 row k sits in lane 32*(k/16) + k%16 (lanes 16-31 of each
//    quarter unused).
//  * Epilogue: 16 warps, four groups of four (one warp per TMEM lane
//    quarter). Group g takes 32-position chunks j = g, g+4, ...; every warp works on
//    its own (channel quarter, chunk) with no barrier between warps. BF16
//    output: 16x256b loads (the accumulator fragment layout: a thread holds
//    two channels x two adjacent positions per 8-column group; for M = 64 the
//    accumulator fills lanes 0-15 of each quarter), position pairs packed to
//    bf16x2 and written with stmatrix.trans as position rows into the warp's
//    own [32 positions][KT/4 channels] staging tile, read back as 16-byte
//    units and stored to y with plain 16-byte stores (positions q >= Q and
//    channels >= K skipped). FP32 output: one channel per thread
//    (32x32b / 16x32bx2 loads), one 32-bit store per value; a warp's store
//    covers consecutive channels of one position (two for M = 64).
//
// Warp roles: warp 0 loads the bands (one thread), warp 1 issues the MMAs
// (one thread), then the epilogue warps (16 for 128-channel tiles, 8 for
// 64-channel tiles: one chunk is a chain of dependent steps, so more warps in
// flight keep the tail of a CTA's last tile short, while fewer leave more
// issue slots to the MMA thread; for 64-channel tiles 8 measured 2.5 %
// faster), then one warp that loads the filter tiles. On GB300 a TMA load
// occupies its issuing thread for roughly 100-250 ns whatever the box size,
// and a single thread issuing bands and filter tiles in turn starved the MMA;
// with two producers and one filter tile per lane the filter stream runs
// ahead of the bands. Bounded waits as in tc_fwd.cu.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int NPOS = 256;  // accumulator columns per tile (largest MMA N)
// Epilogue warps (groups of four lane-quarter warps): 16 for 128-channel
// tiles; 8 for 64-channel tiles, whose epilogue has half the data, so that
// fewer warps share the MMA-issuing thread's sub-partition while the next
// tile's MMAs are issued.
template <int KT>
__host__ __device__ constexpr int epi_warps() { return KT == 64 ? 8 : 16; }
// band producer, MMA issuer, epilogue, filter producer
template <int KT>
__host__ __device__ constexpr int nthreads() { return 96 + 32 * epi_warps<KT>(); }
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 1024;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_SA = 4, MAX_SB = 12;
constexpr int MAX_WRES = 32;  // barriers over the tiles of a resident filter
constexpr int MAX_STRIDE = 4;
constexpr int MAX_PHASES = MAX_STRIDE * MAX_STRIDE;
constexpr int MAX_TAPS = 128;

struct TParams {
    CUtensorMap tmX;  // x [N][H][W][C], box {KE, v*Wx, u*nr, 1}, element strides {1, v, u, 1}
    CUtensorMap tmW;  // w [K][R*S][C], box {KE, 1, KT}
    int N, P, Q, K;
    int u, RS;
    int wx_log2, TR, n_pos;  // n_pos = TR * Wx positions per tile (MMA N)
    int flat;                // 1x1 stride-1 unpadded: x and y as [N*H*W] rows, tiles of n_pos rows
    int M;                   // flat: N*H*W
    // output position (n, p, q) of the P x Q grid is y row
    // (n*out_H + p*ou + oa)*out_W + q*ov + ob (forward: the grid is y itself;
    // data gradient: one sub-pixel phase of dx)
    int out_H, out_W, ou, ov, oa, ob;
    // data gradient: n_ophase > 0 output phases in one launch; phase op owns
    // tiles [op_tile0[op], op_tile0[op+1]), its band origin and taps are phase
    // op of ph_* / tap_*, its grid is op_P x op_Q at offsets (op_oa, op_ob)
    int n_ophase;
    int op_tile0[MAX_PHASES + 1];
    int op_P[MAX_PHASES], op_Q[MAX_PHASES], op_oa[MAX_PHASES], op_ob[MAX_PHASES];
    int op_ptiles[MAX_PHASES];
    // phase f: band origin (column b - pw, row offset a - ph), taps [end[f-1], end[f])
    int n_phase;
    int ph_w0[MAX_PHASES], ph_h0[MAX_PHASES], ph_end[MAX_PHASES];
    uint16_t tap_t[MAX_TAPS];      // filter tap index r*S + s
    uint16_t tap_shift[MAX_TAPS];  // band row offset i*Wx + j
    int c_blocks, k_tiles, p_tiles, num_tiles;
    int band_bytes, band_stride, w_resident, stages_a, stages_b;
    int wgrp;  // streamed filter: tiles per ring stage (stages_b stages)
    int relu, out_f32;
    const float *bias, *x_scale, *w_scale;
    const float *alpha;  // fused per-channel scale (folded batch norm) or null
    const void *z;       // fused residual of y's shape and dtype (may be y) or null
    void *y;  // [N][P][Q][K], BF16 or FP32
    Guard guard;
};

static_assert(sizeof(TParams) <= 4096, "transposed kernel parameters too large");

// One tile: image n, first output row p0 (flat layers: n = 0, p0 = first
// position row), output-channel tile kt, the phases [f0, f1) its bands come
// from, and the P x Q grid and offsets its outputs go to.
struct Tile {
    int n, p0, kt, f0, f1, P, Q, oa, ob;
};

template <bool OPH>
__device__ __forceinline__ Tile tdecode(const TParams &p, int tile) {
    Tile t;
    int lt = tile, ptiles = p.p_tiles;
    t.f0 = 0;
    t.f1 = p.n_phase;
    t.P = p.P;
    t.Q = p.Q;
    t.oa = p.oa;
    t.ob = p.ob;
    if (OPH) {
        int op = 0;
        while (op + 1 < p.n_ophase && tile >= p.op_tile0[op + 1]) ++op;
        lt = tile - p.op_tile0[op];
        ptiles = p.op_ptiles[op];
        t.f0 = op;
        t.f1 = op + 1;
        t.P = p.op_P[op];
        t.Q = p.op_Q[op];
        t.oa = p.op_oa[op];
        t.ob = p.op_ob[op];
    }
    t.kt = lt % p.k_tiles;
    const int mt = lt / p.k_tiles;
    if (p.flat) {
        t.n = 0;
        t.p0 = mt * p.n_pos;
        return t;
    }
    t.n = mt / ptiles;
    t.p0 = (mt - t.n * ptiles) * p.TR;
    return t;
}

// FUSED: the epilogue also applies the per-channel scale and the residual.
// OPH: data-gradient launch, tiles grouped by output phase (n_ophase > 0).
template <int KT, bool FP8, bool FUSED, bool OPH>
__global__ void __launch_bounds__(nthreads<KT>(), 1) tc_fwd_t_kernel(const __grid_constant__ TParams prm) {
    constexpr int EPI_WARPS = epi_warps<KT>();
    constexpr int EPI_GROUPS = EPI_WARPS / 4;
    constexpr int FILTER_WARP = 2 + EPI_WARPS;  // after the epilogue warps
    constexpr int KE = FP8 ? 128 : 64;
    constexpr int TCOLS = 2 * NPOS;          // two 256-column accumulators
    constexpr int W_TILE = KT * 128;         // one filter tile (tap, channel block)
    constexpr int KPW = KT / 4;              // output channels per warp (16 or 32)
    constexpr int NH = KT / 64;              // 16-lane TMEM loads per chunk (BF16 output)
    constexpr int UPR = KPW / 8;             // 16-byte units per staged position row (4 or 2)
    constexpr int SWS = UPR == 4 ? 1 : 2;    // row shift of the staging swizzle
    constexpr int WST = 32 * KPW * 2;        // per-warp staging tile: 32 positions x KPW bf16
    constexpr int EPI_TOTAL = EPI_WARPS * WST;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int SA = prm.stages_a, SB = prm.stages_b;
    const int WG = prm.wgrp;  // streamed filter tiles per stage
    const int w_slots = prm.w_resident ? prm.RS * prm.c_blocks : SB * WG;
    uint8_t *sA = base;                              // band ring
    uint8_t *sW = sA + SA * prm.band_stride;         // filter tiles
    uint8_t *sEpi = sW + w_slots * W_TILE;           // staging
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEpi + EPI_TOTAL);
    uint64_t *fullA = bars;
    uint64_t *emptyA = fullA + MAX_SA;
    uint64_t *fullW = emptyA + MAX_SA;
    uint64_t *emptyW = fullW + MAX_SB;
    uint64_t *tfull = emptyW + MAX_SB;
    uint64_t *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    // Resident filter: tiles stored in the order the MMAs use them (channel
    // block, then tap-table entry), consecutive tiles grouped `wper` to a
    // barrier, so the first MMAs need only the first tiles.
    uint64_t *wres = done + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wres + MAX_WRES);
    const int w_tiles = prm.RS * prm.c_blocks;
    const int wper = (w_tiles + MAX_WRES - 1) / MAX_WRES;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = prm.guard.wait_ns;

    if (threadIdx.x == 0) {
        for (int i = 0; i < SA; ++i) {
            ptx::mbar_init(&fullA[i], 1);
            ptx::mbar_init(&emptyA[i], 1);
        }
        if (prm.w_resident) {
            for (int i = 0; i * wper < w_tiles; ++i) ptx::mbar_init(&wres[i], 1);
        } else {
            for (int i = 0; i < SB; ++i) {
                ptx::mbar_init(&fullW[i], 1);
                ptx::mbar_init(&emptyW[i], 1);
            }
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
        ptx::prefetch_tmap(&prm.tmW);
        // The first tile's bands and filter tiles into L2 while the previous
        // kernel drains (a prefetch fills only L2, which stays coherent with
        // that kernel's writes; the loads come after the dependency wait).
        if ((int)blockIdx.x < prm.num_tiles) {
            const Tile T = tdecode<OPH>(prm, blockIdx.x);
            for (int cb = 0; cb < prm.c_blocks; ++cb)
                for (int f = T.f0; f < T.f1; ++f) {
                    if (prm.flat)
                        ptx::tma_prefetch_2d(&prm.tmX, cb * KE, T.p0);
                    else
                        ptx::tma_prefetch_4d(&prm.tmX, cb * KE, prm.ph_w0[f],
                                             prm.u * T.p0 + prm.ph_h0[f], T.n);
                    for (int ti = f ? prm.ph_end[f - 1] : 0; ti < prm.ph_end[f]; ++ti)
                        ptx::tma_prefetch_3d(&prm.tmW, cb * KE, prm.tap_t[ti],
                                             prm.w_resident ? 0 : T.kt * KT);
                }
        }
    }
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();

    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(prm.guard.err, DEVERR_TIMEOUT);
    };

    if (warp == 0) {
        // ------------------------------ band producer ------------------------------
        if (lane == 0) {
            const bool skip = prm.guard.skip_loads != 0;
            int sa = 0;
            uint32_t pa = 0;
            int issued_a = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x) {
                const Tile T = tdecode<OPH>(prm, tile);
                const int n = T.n, p0 = T.p0;
                for (int cb = 0; ok && cb < prm.c_blocks; ++cb) {
                    for (int f = T.f0; f < T.f1; ++f) {
                        if (!ptx::mbar_wait(&emptyA[sa], pa ^ 1, lim, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        if (!skip) {
                            ptx::mbar_arrive_expect_tx(&fullA[sa], (uint32_t)prm.band_bytes);
                            if (prm.flat)
                                ptx::tma_load_2d(sA + sa * prm.band_stride, &prm.tmX, &fullA[sa],
                                                 cb * KE, p0);
                            else
                                ptx::tma_load_4d(sA + sa * prm.band_stride, &prm.tmX, &fullA[sa],
                                                 cb * KE, prm.ph_w0[f], prm.u * p0 + prm.ph_h0[f], n);
                            ++issued_a;
                        }
                        if (++sa == SA) {
                            sa = 0;
                            pa ^= 1;
                        }
                    }
                }
            }
            volatile int zero = 0;
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
    } else if (warp == FILTER_WARP) {
        // ----------------------------- filter producer -----------------------------
        // Its own warp, so the filter stream runs ahead of the bands by as many
        // tiles as its ring holds. A TMA load costs its issuing thread about as
        // long as a 32 KB box takes to arrive, so the tiles are issued by one
        // lane each, in parallel. All lanes keep the same counters.
        const unsigned FULL = 0xffffffffu;
        const bool skip = prm.guard.skip_loads != 0;
        bool ok = true;
        int issued_w = 0;  // resident filter tiles issued
        long long wq = 0;  // filter tiles that went through the streamed ring
        long long issued_b = 0;
        if (prm.w_resident) {
            // Resident filter: every tile once, in storage order (= MMA order),
            // one per lane; each group's byte count is announced on its barrier
            // (by the lane holding the group's first tile) before any load.
            for (int s0 = 0; !skip && s0 < w_tiles; s0 += 32) {
                const int seq = s0 + lane;
                const bool act = seq < w_tiles;
                if (act && seq % wper == 0) {
                    const int g = seq / wper;
                    ptx::mbar_arrive_expect_tx(&wres[g],
                                               (uint32_t)(min(wper, w_tiles - g * wper) * W_TILE));
                }
                __syncwarp();
                if (act) {
                    const int cb = seq / prm.RS;
                    ptx::tma_load_3d(sW + seq * W_TILE, &prm.tmW, &wres[seq / wper], cb * KE,
                                     prm.tap_t[seq - cb * prm.RS], 0);
                }
                __syncwarp();
            }
            issued_w = skip ? 0 : w_tiles;
        } else {
            // Streamed filter: a tile's filter sequence (channel block, then the
            // taps of its phases) in stages of WG tiles, one barrier pair per
            // stage, one tile per lane; a tile's last stage may be partial.
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x) {
                const Tile T = tdecode<OPH>(prm, tile);
                const int t0 = T.f0 ? prm.ph_end[T.f0 - 1] : 0;
                const int ntp = prm.ph_end[T.f1 - 1] - t0;  // taps per channel block
                const int ntile = prm.c_blocks * ntp;
                for (int j0 = 0; j0 < ntile; j0 += WG, ++wq) {
                    const int cnt = min(WG, ntile - j0);
                    const int stage = (int)(wq % SB);
                    int wok = 1;
                    if (lane == 0) {
                        wok = ptx::mbar_wait(&emptyW[stage], (uint32_t)((wq / SB) & 1) ^ 1u, lim,
                                             abort_flag);
                        if (wok && !skip)
                            ptx::mbar_arrive_expect_tx(&fullW[stage], (uint32_t)(cnt * W_TILE));
                    }
                    if (!__shfl_sync(FULL, wok, 0)) {
                        if (lane == 0) fail();
                        ok = false;
                        break;
                    }
                    if (!skip) {
                        if (lane < cnt) {
                            const int j = j0 + lane, cb = j / ntp;
                            ptx::tma_load_3d(sW + (stage * WG + lane) * W_TILE, &prm.tmW, &fullW[stage],
                                             cb * KE, prm.tap_t[t0 + j - cb * ntp], T.kt * KT);
                        }
                        ++issued_b;
                    }
                }
            }
        }
        if (lane == 0) {
            volatile int zero = 0;
            // the last load of every streamed filter stage
            for (long long i = 1; i <= (issued_b < SB ? issued_b : (long long)SB); ++i) {
                const long long u = wq - i;
                if (!ptx::mbar_wait(&fullW[(int)(u % SB)], (uint32_t)((u / SB) & 1), lim, &zero)) fail();
            }
            // resident filter groups
            for (int b = 0; b * wper < issued_w; ++b)
                if (!ptx::mbar_wait(&wres[b], 0, lim, &zero)) fail();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ----------------------------
            bool ok = true;
            uint32_t idesc = FP8 ? ptx::idesc_e4m3(prm.n_pos) : ptx::idesc_bf16(prm.n_pos);
            idesc = (idesc & ~(0x1Fu << 24)) | ((uint32_t)(KT >> 4) << 24);  // M = KT
            const uint64_t adb = ptx::sdesc_kmajor_sw128(ptx::smem_addr(sW));  // filter slot 0
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            uint32_t wres_seen = 0;  // resident filter groups already waited for
            int local = 0;
            for (int tile = blockIdx.x; ok && tile < prm.num_tiles; tile += gridDim.x, ++local) {
                const int acc = local & 1;
                const uint32_t aph = (local >> 1) & 1;
                if (!ptx::mbar_wait(&tempty[acc], aph ^ 1, lim, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                // only a data-gradient tile restricts the phases; the forward uses all
                int f0 = 0, f1 = prm.n_phase;
                if constexpr (OPH) {
                    const Tile T = tdecode<OPH>(prm, tile);
                    f0 = T.f0;
                    f1 = T.f1;
                }
                const uint32_t d = tmem_base + (uint32_t)(acc * NPOS);
                uint32_t accum = 0;
                // streamed filter: tiles used so far in this tile, and the position
                // inside the current stage of WG tiles
                const int ntile = prm.c_blocks * (prm.ph_end[f1 - 1] - (f0 ? prm.ph_end[f0 - 1] : 0));
                int jw = 0, gi = 0;
                for (int cb = 0; ok && cb < prm.c_blocks; ++cb) {
                    for (int f = f0; f < f1; ++f) {
                        if (!ptx::mbar_wait(&fullA[sa], pa, lim, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        // Descriptors are built once per band; a tap adds its row shift
                        // (128 bytes = 8 descriptor units per row) to the band's and, for a
                        // resident filter, steps one filter tile (tiles are stored in the
                        // order the MMAs use them). The start-address field cannot carry:
                        // shared addresses stay below 256 KB.
                        const uint64_t bdb =
                            ptx::sdesc_kmajor_sw128(ptx::smem_addr(sA + sa * prm.band_stride));
                        const int t0 = f ? prm.ph_end[f - 1] : 0, t1 = prm.ph_end[f];
                        if (prm.w_resident) {
                            const bool first_use = local == 0 || OPH;
                            uint64_t ad = adb + (uint64_t)((cb * prm.RS + t0) * (W_TILE >> 4));
                            for (int ti = t0; ti < t1; ++ti) {
                                if (first_use) {
                                    // the forward's first tile uses every group; a data-gradient
                                    // tile uses its phase's groups, first seen on any tile
                                    const int grp = (cb * prm.RS + ti) / wper;
                                    if (!((wres_seen >> grp) & 1u)) {
                                        if (!ptx::mbar_wait(&wres[grp], 0, lim, abort_flag)) {
                                            fail();
                                            ok = false;
                                            break;
                                        }
                                        ptx::tc_fence_after();
                                        wres_seen |= 1u << grp;
                                    }
                                }
                                const uint64_t bd = bdb + ((uint64_t)prm.tap_shift[ti] << 3);
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    if (FP8)
                                        ptx::mma_f8(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                    else
                                        ptx::mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                    accum = 1;
                                }
                                ad += W_TILE >> 4;
                            }
                        } else {
                            for (int ti = t0; ti < t1; ++ti) {
                                if (gi == 0) {  // first tile of a stage
                                    if (!ptx::mbar_wait(&fullW[sb], pb, lim, abort_flag)) {
                                        fail();
                                        ok = false;
                                        break;
                                    }
                                    ptx::tc_fence_after();
                                }
                                const uint64_t ad = adb + (uint64_t)((sb * WG + gi) * (W_TILE >> 4));
                                const uint64_t bd = bdb + ((uint64_t)prm.tap_shift[ti] << 3);
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    if (FP8)
                                        ptx::mma_f8(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                    else
                                        ptx::mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                    accum = 1;
                                }
                                ++jw;
                                if (++gi == WG || jw == ntile) {  // stage used up
                                    ptx::mma_commit(&emptyW[sb]);
                                    gi = 0;
                                    if (++sb == SB) {
                                        sb = 0;
                                        pb ^= 1;
                                    }
                                }
                            }
                        }
                        if (!ok) break;
                        ptx::mma_commit(&emptyA[sa]);
                        if (++sa == SA) {
                            sa = 0;
                            pa ^= 1;
                        }
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
        const int ew = warp - 2;            // 0..EPI_WARPS-1
        const int quarter = warp & 3;       // TMEM lane quarter
        const int group = ew >> 2;          // chunks j with j % EPI_GROUPS == group
        const int chb0 = quarter * KPW;     // first channel of this warp's lane quarter
        // FP32 output: this thread's channel. KT = 128: lane = channel; KT = 64
        // (two-half loads): lanes l and l+16 share channel l and split the positions
        const int krow = chb0 + (KT == 128 ? lane : (lane & 15));
        uint8_t *wst = sEpi + ew * WST;     // this warp's staging tile
        const int wx_mask = (1 << prm.wx_log2) - 1;
        const float xs = FP8 ? __ldg(prm.x_scale) : 1.f;
        const int nchunks = prm.n_pos >> 5;
        int local = 0;
        for (int tile = blockIdx.x; tile < prm.num_tiles; tile += gridDim.x, ++local) {
            const Tile T = tdecode<OPH>(prm, tile);
            const int n = T.n, p0 = T.p0, kt = T.kt;
            const int acc = local & 1;
            const uint32_t aph = (local >> 1) & 1;
            // per-channel constants, fetched before the accumulator is ready
            float scl = 1.f, bia = 0.f, alf = 1.f;  // FP32 output: channel krow
            float bs[NH][2], ss[NH][2], as[NH][2];  // BF16 output: channels chb0 + 16h + 8s + lane/4
            if (prm.out_f32) {
                const int k = kt * KT + krow;
                if (k < prm.K) {
                    if (FP8) scl = xs * __ldg(prm.w_scale + k);
                    if (prm.bias) bia = __ldg(prm.bias + k);
                    if (FUSED && prm.alpha) alf = __ldg(prm.alpha + k);
                }
            } else {
#pragma unroll
                for (int h = 0; h < NH; ++h)
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const int k = kt * KT + chb0 + 16 * h + 8 * s2 + (lane >> 2);
                        bs[h][s2] = (prm.bias && k < prm.K) ? __ldg(prm.bias + k) : 0.f;
                        ss[h][s2] = (FP8 && k < prm.K) ? xs * __ldg(prm.w_scale + k) : 1.f;
                        as[h][s2] = (FUSED && prm.alpha && k < prm.K) ? __ldg(prm.alpha + k) : 1.f;
                    }
            }
            if constexpr (FUSED) {  // residual of this warp's chunks into L2: lane = position
                if (prm.z) {
                    const int eb = prm.out_f32 ? 4 : 2;
                    const int kw0 = kt * KT + chb0;
                    for (int j = group; j < nchunks && kw0 < prm.K; j += EPI_GROUPS) {
                        size_t row;
                        bool ok;
                        if (prm.flat) {
                            row = (size_t)p0 + 32 * j + lane;
                            ok = row < (size_t)prm.M;
                        } else {
                            const int p = p0 + ((32 * j) >> prm.wx_log2);
                            const int q = ((32 * j) & wx_mask) + lane;
                            ok = p < T.P && q < T.Q;
                            row = ((size_t)n * prm.out_H + (size_t)p * prm.ou + T.oa) * prm.out_W +
                                  T.ob + (size_t)q * prm.ov;
                        }
                        if (ok)
                            ptx::prefetch_l2(static_cast<const char *>(prm.z) +
                                             (row * prm.K + kw0) * eb);
                    }
                }
            }
            if (!ptx::mbar_wait(&tfull[acc], aph, lim, abort_flag)) {
                fail();
                break;
            }
            ptx::tc_fence_after();
            // TMEM load of chunk j into v (not waited for)
            auto tload = [&](int j, uint32_t (&v)[32]) {
                const uint32_t ta = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                    (uint32_t)(acc * NPOS + j * 32);
                if (!prm.out_f32) {
                    // accumulator-fragment layout, 16 channels x 32 positions per load
                    ptx::tmem_ld_16x256b_x4(ta, *reinterpret_cast<uint32_t(*)[16]>(v));
                    if constexpr (KT == 128)
                        ptx::tmem_ld_16x256b_x4(ta + (16u << 16), *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                } else if constexpr (KT == 128) {
                    ptx::tmem_ld_32x32b_x32(ta, *reinterpret_cast<uint32_t(*)[32]>(v));
                } else {
                    ptx::tmem_ld_16x32bx2_x16(ta, *reinterpret_cast<uint32_t(*)[16]>(v));
                }
            };
            // epilogue math and stores of chunk j from v
            auto process = [&](int j, const uint32_t (&v)[32]) {
                size_t yrow;    // y row of the chunk's first position
                size_t ystep;   // y rows between consecutive positions
                int nvalid;     // positions of the chunk inside y
                if (prm.flat) {
                    const int m0 = p0 + 32 * j;
                    if (m0 >= prm.M) return;
                    yrow = (size_t)m0;
                    ystep = 1;
                    nvalid = prm.M - m0;
                } else {
                    const int p = p0 + ((32 * j) >> prm.wx_log2);
                    const int q0 = (32 * j) & wx_mask;
                    if (p >= T.P || q0 >= T.Q) return;
                    yrow = ((size_t)n * prm.out_H + (size_t)p * prm.ou + T.oa) * prm.out_W + T.ob +
                           (size_t)q0 * prm.ov;
                    ystep = (size_t)prm.ov;
                    nvalid = T.Q - q0;
                }
                const int kw = kt * KT + chb0;                                // first channel of the warp
                if (!prm.out_f32) {
                    // Register 4g + 2s (+1) of load h: channel chb0 + 16h + 8s + t/4,
                    // positions 8g + 2(t%4) (+1). Each packed pair is one row of an
                    // 8x8 (channel x position) matrix; stmatrix.trans writes it as 8
                    // position rows of 8 channels (16 bytes) into this warp's
                    // [32 positions][KPW channels] tile. 16-byte units are swizzled
                    // (unit c of row e at c ^ ((e >> SWS) & (UPR - 1))) so that the
                    // eight rows of a matrix and the eight rows read back by a
                    // quarter-warp fall in distinct bank groups.
                    const int mrow = lane & 7, msel = lane >> 3;
                    __syncwarp();  // previous chunk's reads of the tile are done
#pragma unroll
                    for (int h = 0; h < NH; ++h)
#pragma unroll
                        for (int gp = 0; gp < 2; ++gp) {
                            uint32_t pk[4];
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                const int g = 2 * gp + (m >> 1), s2 = m & 1;
                                float a0 = __uint_as_float(v[16 * h + 4 * g + 2 * s2]);
                                float a1 = __uint_as_float(v[16 * h + 4 * g + 2 * s2 + 1]);
                                if (FP8) {
                                    a0 = a0 * ss[h][s2];
                                    a1 = a1 * ss[h][s2];
                                }
                                if (FUSED && prm.alpha) {
                                    a0 = a0 * as[h][s2];
                                    a1 = a1 * as[h][s2];
                                }
                                a0 = a0 + bs[h][s2];
                                a1 = a1 + bs[h][s2];
                                if (FUSED && prm.z) {  // residual of positions e, e+1 of channel kz
                                    const int kz = kw + 16 * h + 8 * s2 + (lane >> 2);
                                    const int e = 8 * g + 2 * (lane & 3);
                                    const __nv_bfloat16 *zp = static_cast<const __nv_bfloat16 *>(prm.z);
                                    if (kz < prm.K) {
                                        if (e < nvalid)
                                            a0 = a0 + __bfloat162float(zp[(yrow + e * ystep) * prm.K + kz]);
                                        if (e + 1 < nvalid)
                                            a1 = a1 + __bfloat162float(
                                                          zp[(yrow + (e + 1) * ystep) * prm.K + kz]);
                                    }
                                }
                                if (prm.relu) {
                                    a0 = fmaxf(a0, 0.f);
                                    a1 = fmaxf(a1, 0.f);
                                }
                                const __nv_bfloat162 b2 = __floats2bfloat162_rn(a0, a1);
                                pk[m] = *reinterpret_cast<const uint32_t *>(&b2);
                            }
                            const int e = 8 * (2 * gp + (msel >> 1)) + mrow;  // position
                            const int c = 2 * h + (msel & 1);                 // 16-byte unit
                            ptx::stmatrix_x4_trans(
                                ptx::smem_addr(wst + e * (UPR * 16) + ((c ^ ((e >> SWS) & (UPR - 1))) << 4)),
                                pk[0], pk[1], pk[2], pk[3]);
                        }
                    __syncwarp();
                    // read back 16-byte units (position e, unit c) and store them to y
#pragma unroll
                    for (int i = 0; i < UPR; ++i) {
                        const int u = i * 32 + lane;
                        const int e = u / UPR, c = u % UPR;
                        const uint4 val = *reinterpret_cast<const uint4 *>(
                            wst + e * (UPR * 16) + ((c ^ ((e >> SWS) & (UPR - 1))) << 4));
                        const int k = kw + 8 * c;
                        if (e < nvalid && k < prm.K)
                            *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(prm.y) +
                                                       (yrow + e * ystep) * prm.K + k) = val;
                    }
                } else {
                    const int k = kt * KT + krow;
                    const int e0 = KT == 128 ? 0 : (lane >> 4) * 16;  // first position of this thread
                    constexpr int NV = KT == 128 ? 32 : 16;
                    float *yf = static_cast<float *>(prm.y);
                    if (k < prm.K) {
#pragma unroll
                        for (int i = 0; i < NV; ++i) {
                            float a = __uint_as_float(v[i]);
                            if (FP8) a = a * scl;
                            if (FUSED && prm.alpha) a = a * alf;
                            a = a + bia;
                            if (e0 + i < nvalid) {
                                const size_t off = (yrow + (e0 + i) * ystep) * prm.K + k;
                                if (FUSED && prm.z) a = a + static_cast<const float *>(prm.z)[off];
                                if (prm.relu) a = fmaxf(a, 0.f);
                                yf[off] = a;
                            }
                        }
                    }
                }
            };
            for (int j = group; j < nchunks; j += EPI_GROUPS) {
                uint32_t v[32];
                tload(j, v);
                ptx::tmem_ld_wait();
                ptx::reg_fence(v);
                if (j + EPI_GROUPS >= nchunks) {  // last TMEM read of this tile by this warp
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                }
                process(j, v);
            }
        }
    }

    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem_base, TCOLS);
}

struct TPlan {
    int wx_log2, TR, nr, band_bytes, band_stride, c_blocks, w_resident, stages_a, stages_b;
    int wgrp;  // streamed filter tiles per ring stage
    int n_phase;
    int flat, n_pos, k_tiles;
    long long num_tiles;
};

bool plan_memory(int kt, long long w_tiles, TPlan *pl, TPlan &p);

// A 1x1, stride-1, unpadded layer is a plain GEMM over the N*H*W positions.
bool is_flat(const Dims &d) {
    return d.R == 1 && d.S == 1 && d.u == 1 && d.v == 1 && d.ph == 0 && d.pw == 0;
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

template <int KT>
constexpr int epi_total() { return epi_warps<KT>() * 32 * (KT / 4) * 2; }  // per-warp staging tiles

// Largest band shift of the phase decomposition: i = (r*dh) div u over the
// rows, j = (s*dw) div v over the columns.
int max_shift(int taps, int dil, int stride) { return ((taps - 1) * dil) / stride; }

int count_phases(const Dims &d) {
    bool used[MAX_PHASES] = {};
    int n = 0;
    for (int r = 0; r < d.R; ++r)
        for (int s = 0; s < d.S; ++s) {
            const int f = ((r * d.dh) % d.u) * d.v + (s * d.dw) % d.v;
            if (!used[f]) {
                used[f] = true;
                ++n;
            }
        }
    return n;
}

bool make_plan(const Dims &d, int kt, TPlan *pl) {
    if (d.u > MAX_STRIDE || d.v > MAX_STRIDE || d.R * d.S > MAX_TAPS) return false;
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    const int ke = fp8 ? 128 : 64;
    const int k_tiles = (d.K + kt - 1) / kt;
    TPlan p{};
    p.k_tiles = k_tiles;
    p.c_blocks = (d.C + ke - 1) / ke;
    if (is_flat(d)) {
        // Tiles of n_pos consecutive positions; n_pos (a multiple of 32, 128..256)
        // minimises the rounds of tiles over the SMs, each round costing its
        // positions plus about 32 positions' worth of per-tile overhead.
        const long long M = d.M();
        const int sms = sm_count();
        long long best = -1;
        for (int np = 256; np >= 128; np -= 32) {
            const long long tiles = (M + np - 1) / np * k_tiles;
            const long long cost = (tiles + sms - 1) / sms * (np + 32);
            if (best < 0 || cost < best) {
                best = cost;
                p.n_pos = np;
            }
        }
        p.flat = 1;
        p.wx_log2 = 0;
        p.TR = 1;
        p.nr = 1;
        p.n_phase = 1;
        p.num_tiles = (M + p.n_pos - 1) / p.n_pos * k_tiles;
        p.band_bytes = 128 * p.n_pos;
        p.band_stride = (p.band_bytes + 1023) / 1024 * 1024;
    } else {
        const int imax = max_shift(d.R, d.dh, d.u), jmax = max_shift(d.S, d.dw, d.v);
        const int need = d.Q + jmax;
        int wx = 32;
        while (wx < need) wx *= 2;
        if (wx > NPOS || wx * d.v > 256) return false;  // TMA box extent <= 256
        p.wx_log2 = ilog2(wx);
        // rows per tile: at most 256 / Wx, spread evenly over the output rows
        const int tr_max = NPOS / wx;
        const int row_tiles = std::max(1, (d.P + tr_max - 1) / tr_max);
        p.TR = std::max(1, (d.P + row_tiles - 1) / row_tiles);
        p.nr = p.TR + imax;
        if (p.nr * d.u > 256) return false;
        p.band_bytes = 128 * wx * p.nr;
        p.band_stride = (p.band_bytes + jmax * 128 + 1023) / 1024 * 1024;
        if (p.band_stride > 80 * 1024) return false;
        p.n_phase = count_phases(d);
        p.num_tiles = (long long)d.N * ((d.P + p.TR - 1) / p.TR) * k_tiles;
        p.n_pos = p.TR << p.wx_log2;
    }
    return plan_memory(kt, (long long)d.R * d.S * p.c_blocks, pl, p);
}

// Shared-memory split of a plan whose geometry (band size, channel blocks,
// channel tiles) is set: the filter resident when there is one channel tile
// and it fits beside two bands, else streamed through a ring of tiles.
bool plan_memory(int kt, long long w_tiles, TPlan *pl, TPlan &p) {
    const int epi = kt == 128 ? epi_total<128>() : epi_total<64>();
    const int budget = SMEM_LIMIT - SMEM_ALIGN - BAR_BYTES - epi;
    const int wtile = kt * 128;
    const long long w_total = w_tiles * wtile;
    if (p.k_tiles == 1 && w_total + 2ll * p.band_stride <= budget) {
        p.w_resident = 1;
        p.stages_a = (int)std::min<long long>(MAX_SA, (budget - w_total) / p.band_stride);
        p.stages_b = 0;
        p.wgrp = 1;
    } else {
        // a third band stage when the filter ring keeps at least 4 slots: a band
        // comes from HBM, a filter tile from L2, so bands need the longer lead
        p.w_resident = 0;
        p.stages_a = (budget - 3 * p.band_stride) / wtile >= 4 ? 3 : 2;
        const int slots = std::min(MAX_SB, (budget - p.stages_a * p.band_stride) / wtile);
        if (slots < 2) return false;
        // stages of up to 4 tiles (one barrier wait and one commit per stage on
        // the MMA thread), at least two stages
        p.wgrp = slots >= 8 ? 4 : slots >= 6 ? 3 : slots >= 4 ? 2 : 1;
        p.stages_b = slots / p.wgrp;
    }
    *pl = p;
    return true;
}

// Tap table: taps grouped by phase (a, b), phases in order f = a*v + b,
// phases without taps left out.
void build_taps(const Dims &d, int wx_log2, TParams *prm) {
    int n = 0, f_out = 0;
    for (int a = 0; a < d.u; ++a)
        for (int b = 0; b < d.v; ++b) {
            const int start = n;
            for (int r = 0; r < d.R; ++r) {
                if ((r * d.dh) % d.u != a) continue;
                for (int s = 0; s < d.S; ++s) {
                    if ((s * d.dw) % d.v != b) continue;
                    const int i = (r * d.dh) / d.u, j = (s * d.dw) / d.v;
                    prm->tap_t[n] = (uint16_t)(r * d.S + s);
                    prm->tap_shift[n] = (uint16_t)((i << wx_log2) + j);
                    ++n;
                }
            }
            if (n == start) continue;
            prm->ph_w0[f_out] = b - d.pw;
            prm->ph_h0[f_out] = a - d.ph;
            prm->ph_end[f_out] = n;
            ++f_out;
        }
    prm->n_phase = f_out;
}

template <int KT, bool FP8, bool FUSED, bool OPH>
gbconv_status_t launch_one(const TParams &prm, size_t smem, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fwd_t_kernel<KT, FP8, FUSED, OPH>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    return cuda_status(
        launch_pdl(tc_fwd_t_kernel<KT, FP8, FUSED, OPH>, dim3(grid), dim3(nthreads<KT>()), smem, st, prm));
}

// forward launches (with or without the fused epilogue)
template <int KT, bool FP8>
gbconv_status_t launch(const TParams &prm, size_t smem, int grid, cudaStream_t st) {
    return (prm.alpha || prm.z) ? launch_one<KT, FP8, true, false>(prm, smem, grid, st)
                                : launch_one<KT, FP8, false, false>(prm, smem, grid, st);
}

}  // namespace

// Output-channel tile of the transposed kernel for this layer (0 if none fits).
int tc_fwd_t_tile(const Dims &d) {
    if (!tc_fwd_supported(d)) return 0;
    // K > 128: a band is fetched once per 128-channel tile (automatic choice
    // only when the filter could not stay resident in the pixel-major band kernel)
    const int kt = d.K <= 64 ? 64 : 128;
    TPlan p;
    return make_plan(d, kt, &p) ? kt : 0;
}

gbconv_status_t launch_tc_fwd_t(const Dims &d, const void *x, const void *w, const float *bias,
                                const float *x_scale, const float *w_scale, void *y,
                                cudaStream_t st, const Fused &fz) {
    const int kt = tc_fwd_t_tile(d);
    if (!kt) return GBCONV_ERR_UNSUPPORTED;
    TPlan pl;
    make_plan(d, kt, &pl);
    if (d.M() == 0) return GBCONV_OK;
    const bool fp8 = d.in_dtype == GBCONV_E4M3;
    const int eb = fp8 ? 1 : 2, ke = 128 / eb;
    const CUtensorMapDataType in_t =
        fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    TParams prm;
    memset(&prm, 0, sizeof(prm));
    gbconv_status_t s;
    if (pl.flat) {  // x as [N*H*W][C], boxes of n_pos rows
        uint64_t xd[2] = {(uint64_t)d.C, (uint64_t)d.M()};
        uint64_t xs[1] = {(uint64_t)d.C * eb};
        uint32_t xb[2] = {(uint32_t)ke, (uint32_t)pl.n_pos};
        s = encode_tiled(&prm.tmX, in_t, 2, x, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_128B);
    } else {
        uint64_t xd[4] = {(uint64_t)d.C, (uint64_t)d.W, (uint64_t)d.H, (uint64_t)d.N};
        uint64_t xs[3] = {(uint64_t)d.C * eb, (uint64_t)d.W * d.C * eb,
                          (uint64_t)d.H * d.W * d.C * eb};
        uint32_t xb[4] = {(uint32_t)ke, (uint32_t)(d.v << pl.wx_log2), (uint32_t)(d.u * pl.nr), 1};
        uint32_t xe[4] = {1, (uint32_t)d.v, (uint32_t)d.u, 1};
        s = encode_tiled(&prm.tmX, in_t, 4, x, xd, xs, xb, CU_TENSOR_MAP_SWIZZLE_128B, xe);
    }
    if (s != GBCONV_OK) return s;
    uint64_t wd[3] = {(uint64_t)d.C, (uint64_t)d.R * d.S, (uint64_t)d.K};
    uint64_t wstr[2] = {(uint64_t)d.C * eb, (uint64_t)d.R * d.S * d.C * eb};
    uint32_t wbx[3] = {(uint32_t)ke, 1, (uint32_t)kt};
    s = encode_tiled(&prm.tmW, in_t, 3, w, wd, wstr, wbx, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    const bool of32 = d.out_dtype == GBCONV_F32;
    if (reinterpret_cast<uintptr_t>(y) % 16) return GBCONV_ERR_ALIGNMENT;  // 16-byte stores
    prm.y = y;
    prm.N = d.N;
    prm.P = d.P;
    prm.Q = d.Q;
    prm.out_H = d.P;
    prm.out_W = d.Q;
    prm.ou = prm.ov = 1;
    prm.oa = prm.ob = 0;
    prm.K = d.K;
    prm.u = d.u;
    prm.RS = d.R * d.S;
    prm.wx_log2 = pl.wx_log2;
    build_taps(d, pl.wx_log2, &prm);
    prm.TR = pl.TR;
    prm.n_pos = pl.n_pos;
    prm.flat = pl.flat;
    prm.M = (int)d.M();
    prm.c_blocks = pl.c_blocks;
    prm.k_tiles = pl.k_tiles;
    prm.p_tiles = (d.P + pl.TR - 1) / pl.TR;
    if (pl.num_tiles >= (1ll << 31)) return GBCONV_ERR_UNSUPPORTED;
    prm.num_tiles = (int)pl.num_tiles;
    prm.band_bytes = pl.band_bytes;
    prm.band_stride = pl.band_stride;
    prm.w_resident = pl.w_resident;
    prm.stages_a = pl.stages_a;
    prm.stages_b = pl.stages_b;
    prm.wgrp = pl.wgrp;
    prm.relu = (d.flags & GBCONV_FLAG_RELU) ? 1 : 0;
    prm.out_f32 = of32;
    prm.bias = (d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr;
    prm.x_scale = x_scale;
    prm.w_scale = w_scale;
    prm.alpha = fz.alpha;
    prm.z = fz.z;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const int w_slots = pl.w_resident ? d.R * d.S * pl.c_blocks : pl.stages_b * pl.wgrp;
    const size_t smem = (size_t)SMEM_ALIGN + (size_t)pl.stages_a * pl.band_stride +
                        (size_t)w_slots * kt * 128 +
                        (kt == 128 ? epi_total<128>() : epi_total<64>()) + BAR_BYTES;
    const int grid = std::min(prm.num_tiles, sm_count());
    if (kt == 64) return fp8 ? launch<64, true>(prm, smem, grid, st) : launch<64, false>(prm, smem, grid, st);
    return fp8 ? launch<128, true>(prm, smem, grid, st) : launch<128, false>(prm, smem, grid, st);
}

// ---------------------------------------------------------------------------
// Data gradient of a strided layer by sub-pixel phases (the transposed
// convolution of the backward pass, paper Sec. 5.B):
//
//   dx[n, u*h' + a, v*w' + b, c] = sum_{k, r in R_a, s in S_b}
//       dy[n, h' + off_r, w' + off_s, k] * w[k, r, s, c]
//
// with R_a = {r : (a + ph - r*dh) divisible by u}, off_r = (a + ph - r*dh) / u
// (S_b, off_s likewise). Each output phase (a, b) is a stride-1 correlation of
// dy with the taps of R_a x S_b at offsets (off_r, off_s); it runs on the band
// kernel with dy as input (K channels), the filter transposed to
// wT[c][r*S + s][k], and the output positions scattered to dx rows
// u*h' + a, columns v*w' + b. Phases without taps are zero.

namespace {

struct PhaseTaps {
    int n;                      // taps
    int off_min_r, off_max_r, off_min_s, off_max_s;
    int t[MAX_TAPS], off_r[MAX_TAPS], off_s[MAX_TAPS];
};

void phase_taps(const Dims &d, int a, int b, PhaseTaps *pt) {
    pt->n = 0;
    pt->off_min_r = pt->off_min_s = 1 << 30;
    pt->off_max_r = pt->off_max_s = -(1 << 30);
    for (int r = 0; r < d.R; ++r) {
        const int nr = a + d.ph - r * d.dh;
        if (((nr % d.u) + d.u) % d.u) continue;
        for (int s = 0; s < d.S; ++s) {
            const int ns = b + d.pw - s * d.dw;
            if (((ns % d.v) + d.v) % d.v) continue;
            const int orr = nr / d.u, os = ns / d.v;  // exact (possibly negative) quotients
            pt->t[pt->n] = r * d.S + s;
            pt->off_r[pt->n] = orr;
            pt->off_s[pt->n] = os;
            pt->off_min_r = std::min(pt->off_min_r, orr);
            pt->off_max_r = std::max(pt->off_max_r, orr);
            pt->off_min_s = std::min(pt->off_min_s, os);
            pt->off_max_s = std::max(pt->off_max_s, os);
            ++pt->n;
        }
    }
}

// All output phases of one data gradient, in one launch: common band shape
// (Wx, TR, nr over the widest phase), phases with more taps first so their
// longer tiles start early.
struct DgradPlan {
    TPlan pl;
    int n_op;                          // phases with taps
    int a[MAX_PHASES], b[MAX_PHASES];  // their offsets, in launch order
    int Ha[MAX_PHASES], Wb[MAX_PHASES];
    PhaseTaps taps[MAX_PHASES];
    int n_zero;                        // phases no tap reaches
    int za[MAX_PHASES], zb[MAX_PHASES];
};

int dgrad_tile(const Dims &d) { return d.C <= 64 ? 64 : 128; }

bool dgrad_plan(const Dims &d, DgradPlan *dp) {
    if (d.u > MAX_STRIDE || d.v > MAX_STRIDE || d.R * d.S > MAX_TAPS) return false;
    const int kt = dgrad_tile(d), ke = 64;  // BF16
    dp->n_op = dp->n_zero = 0;
    int ispan = 0, jspan = 0, wneed = 0, hmax = 0;
    for (int a = 0; a < std::min(d.u, d.H); ++a)
        for (int b = 0; b < std::min(d.v, d.W); ++b) {
            PhaseTaps &pt = dp->taps[dp->n_op];
            phase_taps(d, a, b, &pt);
            if (pt.n == 0) {
                dp->za[dp->n_zero] = a;
                dp->zb[dp->n_zero] = b;
                ++dp->n_zero;
                continue;
            }
            const int Ha = (d.H - a + d.u - 1) / d.u, Wb = (d.W - b + d.v - 1) / d.v;
            dp->a[dp->n_op] = a;
            dp->b[dp->n_op] = b;
            dp->Ha[dp->n_op] = Ha;
            dp->Wb[dp->n_op] = Wb;
            ispan = std::max(ispan, pt.off_max_r - pt.off_min_r);
            jspan = std::max(jspan, pt.off_max_s - pt.off_min_s);
            wneed = std::max(wneed, Wb + pt.off_max_s - pt.off_min_s);
            hmax = std::max(hmax, Ha);
            ++dp->n_op;
        }
    // longest phases (most taps) first: a stable insertion sort of the phases
    for (int i = 1; i < dp->n_op; ++i)
        for (int j = i; j > 0 && dp->taps[j].n > dp->taps[j - 1].n; --j) {
            std::swap(dp->taps[j], dp->taps[j - 1]);
            std::swap(dp->a[j], dp->a[j - 1]);
            std::swap(dp->b[j], dp->b[j - 1]);
            std::swap(dp->Ha[j], dp->Ha[j - 1]);
            std::swap(dp->Wb[j], dp->Wb[j - 1]);
        }
    if (dp->n_op == 0) return true;
    int wx = 32;
    while (wx < wneed) wx *= 2;
    if (wx > NPOS) return false;
    TPlan &p = dp->pl;
    p = TPlan{};
    p.k_tiles = (d.C + kt - 1) / kt;
    p.c_blocks = (d.K + ke - 1) / ke;
    p.wx_log2 = ilog2(wx);
    const int tr_max = NPOS / wx;
    const int row_tiles = std::max(1, (hmax + tr_max - 1) / tr_max);
    p.TR = std::max(1, (hmax + row_tiles - 1) / row_tiles);
    p.nr = p.TR + ispan;
    if (p.nr > 256) return false;
    p.band_bytes = 128 * wx * p.nr;
    p.band_stride = (p.band_bytes + jspan * 128 + 1023) / 1024 * 1024;
    if (p.band_stride > 80 * 1024) return false;
    p.n_phase = dp->n_op;
    p.n_pos = p.TR << p.wx_log2;
    long long tiles = 0, taps = 0;
    for (int i = 0; i < dp->n_op; ++i) {
        tiles += (long long)d.N * ((dp->Ha[i] + p.TR - 1) / p.TR) * p.k_tiles;
        taps += dp->taps[i].n;
    }
    if (taps > MAX_TAPS || tiles >= (1ll << 31)) return false;
    p.num_tiles = tiles;
    TPlan out;
    if (!plan_memory(kt, taps * p.c_blocks, &out, p)) return false;
    p = out;
    return true;
}

}  // namespace

bool tc_dgrad_t_supported(const Dims &d) {
    if (d.layout != GBCONV_NHWC || d.in_dtype != GBCONV_BF16) return false;
    if (d.out_dtype != GBCONV_BF16 && d.out_dtype != GBCONV_F32) return false;
    if (d.C % 8 || d.K % 8) return false;
    if (d.M() >= (1ll << 31) || (long long)d.N * d.H * d.W >= (1ll << 31)) return false;
    DgradPlan dp;
    return dgrad_plan(d, &dp);
}

gbconv_status_t launch_tc_dgrad_t(const Dims &d, const void *dy, const void *wT, void *dx,
                                  cudaStream_t st) {
    if (!tc_dgrad_t_supported(d)) return GBCONV_ERR_UNSUPPORTED;
    if ((long long)d.N * d.H * d.W == 0) return GBCONV_OK;
    if (reinterpret_cast<uintptr_t>(dx) % 16) return GBCONV_ERR_ALIGNMENT;
    DgradPlan dp;
    dgrad_plan(d, &dp);
    for (int i = 0; i < dp.n_zero; ++i) {  // positions no tap reaches
        gbconv_status_t s = launch_zero_phase(d, dx, dp.za[i], dp.zb[i], st);
        if (s != GBCONV_OK) return s;
    }
    if (dp.n_op == 0) return GBCONV_OK;
    const TPlan &pl = dp.pl;
    const int kt = dgrad_tile(d);
    const int ke = 64, eb = 2;
    TParams prm;
    memset(&prm, 0, sizeof(prm));
    // dy [N][P][Q][K]: bands of nr rows x Wx columns, stride 1
    uint64_t xd[4] = {(uint64_t)d.K, (uint64_t)d.Q, (uint64_t)d.P, (uint64_t)d.N};
    uint64_t xs[3] = {(uint64_t)d.K * eb, (uint64_t)d.Q * d.K * eb, (uint64_t)d.P * d.Q * d.K * eb};
    uint32_t xb[4] = {(uint32_t)ke, (uint32_t)(1 << pl.wx_log2), (uint32_t)pl.nr, 1};
    gbconv_status_t s = encode_tiled(&prm.tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, dy, xd, xs, xb,
                                     CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    // wT [C][R*S][K]
    uint64_t wd[3] = {(uint64_t)d.K, (uint64_t)d.R * d.S, (uint64_t)d.C};
    uint64_t wstr[2] = {(uint64_t)d.K * eb, (uint64_t)d.R * d.S * d.K * eb};
    uint32_t wbx[3] = {(uint32_t)ke, 1, (uint32_t)kt};
    s = encode_tiled(&prm.tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, wT, wd, wstr, wbx,
                     CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    prm.y = dx;
    prm.N = d.N;
    prm.K = d.C;
    prm.out_H = d.H;
    prm.out_W = d.W;
    prm.ou = d.u;
    prm.ov = d.v;
    prm.u = 1;
    prm.wx_log2 = pl.wx_log2;
    prm.n_phase = dp.n_op;
    prm.n_ophase = dp.n_op;
    int nt = 0, tile0 = 0;
    for (int op = 0; op < dp.n_op; ++op) {
        const PhaseTaps &pt = dp.taps[op];
        prm.ph_w0[op] = pt.off_min_s;
        prm.ph_h0[op] = pt.off_min_r;
        for (int i = 0; i < pt.n; ++i, ++nt) {
            prm.tap_t[nt] = (uint16_t)pt.t[i];
            prm.tap_shift[nt] = (uint16_t)(((pt.off_r[i] - pt.off_min_r) << pl.wx_log2) +
                                           (pt.off_s[i] - pt.off_min_s));
        }
        prm.ph_end[op] = nt;
        prm.op_P[op] = dp.Ha[op];
        prm.op_Q[op] = dp.Wb[op];
        prm.op_oa[op] = dp.a[op];
        prm.op_ob[op] = dp.b[op];
        prm.op_ptiles[op] = (dp.Ha[op] + pl.TR - 1) / pl.TR;
        prm.op_tile0[op] = tile0;
        tile0 += d.N * prm.op_ptiles[op] * pl.k_tiles;
    }
    prm.op_tile0[dp.n_op] = tile0;
    prm.RS = nt;
    prm.TR = pl.TR;
    prm.n_pos = pl.n_pos;
    prm.c_blocks = pl.c_blocks;
    prm.k_tiles = pl.k_tiles;
    prm.num_tiles = (int)pl.num_tiles;
    prm.band_bytes = pl.band_bytes;
    prm.band_stride = pl.band_stride;
    prm.w_resident = pl.w_resident;
    prm.stages_a = pl.stages_a;
    prm.stages_b = pl.stages_b;
    prm.wgrp = pl.wgrp;
    prm.out_f32 = d.out_dtype == GBCONV_F32;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const int w_slots = pl.w_resident ? nt * pl.c_blocks : pl.stages_b * pl.wgrp;
    const size_t smem = (size_t)SMEM_ALIGN + (size_t)pl.stages_a * pl.band_stride +
                        (size_t)w_slots * kt * 128 +
                        (kt == 128 ? epi_total<128>() : epi_total<64>()) + BAR_BYTES;
    const int grid = std::min(prm.num_tiles, sm_count());
    return kt == 64 ? launch_one<64, false, false, true>(prm, smem, grid, st)
                    : launch_one<128, false, false, true>(prm, smem, grid, st);
}

}  // namespace gbc
