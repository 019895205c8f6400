// tc_wgrad_shift.cu -- tensor-core (tcgen05) weight gradient of stride-1 NHWC
// BF16 layers, the filter taps of one filter row taken as row shifts of one
// input band (paper Sec. 5.B, backward pass of a convolutional layer):
//
//   dw[k, r, s, c] = sum_{n,p,q} dy[n, p, q, k] * x[n, p - ph + r*dh, q - pw + s*dw, c]
//
// A work unit is (slice, 128-channel output tile, filter row r, BN-channel
// input tile). Its reduction runs over "bands" of TR consecutive output rows
// of one image, each row laid out as Wx >= Q pixel positions (dy is zero at
// positions q >= Q). Per band the producers load, MN-major (one 128-byte row
// of 64 channels per pixel position):
//   dy band: TR x Wx positions of 128 output channels (two 64-channel boxes);
//   x band:  input rows p - ph + r*dh and columns -pw .. Wx - pw - 1 of the same
//            TR rows, BN input channels (BN / 64 boxes).
// With j the band position of output pixel (t, q) (j = t*Wx + q), the input
// pixel of tap s sits at band position j + s*dw, so tap s is the GEMM
//   D_s[k][c] += sum_j dy_band[j][k] * x_band[j + s*dw][c],
// one MMA chain reading the x band from a start row s*dw further on. The S
// accumulators of filter row r (S * BN TMEM columns) stay resident for the
// whole unit: dy and x reach the SM once per filter row instead of once per
// tap (for 3x3 layers a third of the per-tap kernel's shared-memory ingest).
//
// Row width. Wx = Q + max(0, (S-1)*dw - pw). Positions q + s*dw >= Wx (needed
// only when the right padding covers them) spill into the first positions of
// the next band row, which hold input columns < 0: zero, as the correct value
// (an input column >= W) is. On the last band row they spill past the box into
// shared-memory rows that are zeroed once and never written by TMA; the same
// zero rows pad each band to a multiple of 16 positions (the MMA's K).
//
// The slices' FP32 partial tiles leave through 4-D TMA stores into the
// workspace [slice][K][R*S][C]; the slice sum is the same fixed-order
// compensated reduction as for the per-tap kernel.
//
// Warp roles (288 threads): warps 0 and 6-8 producers (bands taken in turn,
// one box per lane), warp 1 TMEM allocation and MMA issue (one thread), warps
// 2-5 epilogue (one TMEM lane quarter each). All waits are bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace gbc {
namespace {

constexpr int KT = 128;            // output-channel tile = MMA M
constexpr int NPROD = 4;           // producer warps: 0 and 6 .. 4 + NPROD
constexpr int NTHREADS = 64 + 32 * 4 + 32 * (NPROD - 1);
constexpr int EPI_WARPS = 4;
constexpr int EPI_BYTES = 8192;    // two 4 KB FP32 chunk buffers per epilogue warp
constexpr int EPI_TOTAL = EPI_WARPS * EPI_BYTES;
constexpr int SMEM_ALIGN = 1024;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_STAGES = 8;
constexpr int SMS_FOR_DEFAULTS = 152;  // split heuristic (host-only, no device query)

// Band geometry of one layer (host-chosen, see plan()).
struct Plan {
    int bn;        // input-channel tile (64 or 128)
    int wx;        // positions per band row
    int tr;        // output rows per band
    int jpad;      // band positions rounded up to 16
    int xrows;     // x band rows allocated (jpad + (S-1)*dw, rounded up to 8)
    int a_blk;     // bytes of one 64-channel dy block
    int b_blk;     // bytes of one 64-channel x block
    int stages;
    int bpi;       // bands per image
    int acc_cols;  // TMEM columns of one accumulator set (S * bn)
    int nacc;      // accumulator sets (1 or 2)
    int tcols;     // TMEM columns allocated (power of two)
};

struct WsParams {
    CUtensorMap tmG;  // dy [N][P][Q][K], box 64 x Wx x TR x 1
    CUtensorMap tmX;  // x  [N][H][W][C], box 64 x Wx x TR x 1
    CUtensorMap tmW;  // partials [slices][K][R*S][C], FP32
    int K, S, dw, ph, pw, dh;
    int tr, bpi, nbands, ksteps, valid_rows, xrows, jpad;
    int a_blk, b_blk, stages, acc_cols, nacc, tcols;
    int nprod;  // producer warps in use: min(NPROD, stages)
    int k_tiles, c_tiles, R, slices, units;
    Guard guard;
};

__device__ __forceinline__ void unit_decode(const WsParams &p, int u, int &slice, int &kt, int &r,
                                            int &ct) {
    ct = u % p.c_tiles;
    int t = u / p.c_tiles;
    r = t % p.R;
    t /= p.R;
    kt = t % p.k_tiles;
    slice = t / p.k_tiles;
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1) tc_wgrad_shift_kernel(const __grid_constant__ WsParams prm) {
    constexpr int XB = BN / 64;  // x boxes per band
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + SMEM_ALIGN - 1) & ~uintptr_t(SMEM_ALIGN - 1));
    const int stages = prm.stages;
    const int a_stage = 2 * prm.a_blk, b_stage = XB * prm.b_blk;
    uint8_t *sA = base;
    uint8_t *sB = base + stages * a_stage;
    uint8_t *sEpi = sB + stages * b_stage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEpi + EPI_TOTAL);
    uint64_t *full = bars;
    uint64_t *empty = bars + MAX_STAGES;
    uint64_t *tfull = bars + 2 * MAX_STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *done = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = prm.guard.wait_ns;

    // Zero the shared-memory rows that TMA never writes: the band's padding
    // to 16 positions (dy and x) and the rows past the x box that the shifted
    // taps of the last band row read.
    {
        const int vrow = prm.valid_rows;
        const int a_words = (prm.jpad - vrow) * 8, b_words = (prm.xrows - vrow) * 8;  // 16-byte words
        const int per_stage = 2 * a_words + XB * b_words;
        for (int i = threadIdx.x; i < stages * per_stage; i += NTHREADS) {
            const int st = i / per_stage;
            int w = i - st * per_stage;
            uint8_t *p;
            if (w < 2 * a_words) {
                const int blk = w / a_words;
                w -= blk * a_words;
                p = sA + st * a_stage + blk * prm.a_blk + vrow * 128 + w * 16;
            } else {
                w -= 2 * a_words;
                const int blk = w / b_words;
                w -= blk * b_words;
                p = sB + st * b_stage + blk * prm.b_blk + vrow * 128 + w * 16;
            }
            *reinterpret_cast<uint4 *>(p) = make_uint4(0u, 0u, 0u, 0u);
        }
        ptx::fence_proxy_async_smem();
    }
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
        ptx::tmem_alloc(tmem_slot, (uint32_t)prm.tcols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (threadIdx.x == 0) {
        ptx::prefetch_tmap(&prm.tmG);
        ptx::prefetch_tmap(&prm.tmX);
        ptx::prefetch_tmap(&prm.tmW);
    }
    ptx::griddep_wait();
    if (threadIdx.x == 0) ptx::griddep_launch();

    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(prm.guard.err, DEVERR_TIMEOUT);
    };
    auto band_range = [&](int slice, int &b0, int &b1) {
        b0 = (int)((long long)prm.nbands * slice / prm.slices);
        b1 = (int)((long long)prm.nbands * (slice + 1) / prm.slices);
    };

    if (warp == 0 || warp >= 6) {
        // ------------------------------ producers ------------------------------
        // Band `it` of this CTA is issued by producer warp it % nprod (one box
        // per lane); nprod <= stages keeps each ring-slot wait on the slot's
        // previous use.
        const unsigned FULL = 0xffffffffu;
        const int me = warp == 0 ? 0 : warp - 5;
        const bool skip = prm.guard.skip_loads != 0;
        const uint32_t bytes = (uint32_t)(2 + XB) * (uint32_t)prm.valid_rows * 128u;
        long long it = 0;     // bands of this CTA so far (all producer warps)
        long long last = -1;  // last band this warp issued
        bool ok = me < prm.nprod;
        for (int u = blockIdx.x; ok && u < prm.units; u += gridDim.x) {
            int slice, kt, r, ct, b0, b1;
            unit_decode(prm, u, slice, kt, r, ct);
            band_range(slice, b0, b1);
            const int xh = -prm.ph + r * prm.dh;  // input row of output row 0
            for (int b = b0; b < b1; ++b, ++it) {
                if ((int)(it % prm.nprod) != me) continue;
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
                const int n = b / prm.bpi, p0 = (b - n * prm.bpi) * prm.tr;
                if (lane < 2) {
                    ptx::tma_load_4d(sA + stage * a_stage + lane * prm.a_blk, &prm.tmG, &full[stage],
                                     kt * KT + 64 * lane, 0, p0, n);
                } else if (lane < 2 + XB) {
                    const int j = lane - 2;
                    ptx::tma_load_4d(sB + stage * b_stage + j * prm.b_blk, &prm.tmX, &full[stage],
                                     ct * BN + 64 * j, -prm.pw, p0 + xh, n);
                }
                last = it;
            }
        }
        // this warp's bands among the CTA's last `stages` may still be in flight
        if (lane == 0 && !skip) {
            volatile int zero = 0;
            for (long long j = last; j >= 0 && j >= it - stages; j -= prm.nprod)
                if (!ptx::mbar_wait(&full[(int)(j % stages)], (uint32_t)((j / stages) & 1), lim, &zero))
                    fail();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ----------------------------
            // MN-major operands: 64-channel blocks a_blk / b_blk bytes apart;
            // one K step of 16 positions is 16 rows = 2048 B; tap s starts the
            // x operand s*dw rows (128 B each) further on.
            const uint32_t idesc = ptx::idesc_bf16(BN, 1, 1);
            const int S = prm.S, ksteps = prm.ksteps;
            const uint32_t tap_step = (uint32_t)(prm.dw * 128) >> 4;
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            for (int u = blockIdx.x; ok && u < prm.units; u += gridDim.x, ++local) {
                int slice, kt, r, ct, b0, b1;
                unit_decode(prm, u, slice, kt, r, ct);
                band_range(slice, b0, b1);
                const int acc = prm.nacc == 2 ? (local & 1) : 0;
                const uint32_t aph = (uint32_t)((prm.nacc == 2 ? local >> 1 : local) & 1);
                if (!ptx::mbar_wait(&tempty[acc], aph ^ 1, lim, abort_flag)) {
                    fail();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d0 = tmem_base + (uint32_t)(acc * prm.acc_cols);
                for (int b = b0; b < b1; ++b) {
                    if (!ptx::mbar_wait(&full[stage], phase, lim, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t ad =
                        ptx::sdesc_mnmajor_sw128(ptx::smem_addr(sA + stage * a_stage), prm.a_blk);
                    const uint64_t bd =
                        ptx::sdesc_mnmajor_sw128(ptx::smem_addr(sB + stage * b_stage), prm.b_blk);
                    for (int k = 0; k < ksteps; ++k) {
                        const uint32_t acc_in = (b > b0 || k > 0) ? 1u : 0u;
                        const uint64_t ak = ad + (uint64_t)(k * 128);  // 2048 B >> 4
                        for (int s = 0; s < S; ++s)
                            ptx::mma_f16(d0 + (uint32_t)(s * BN), ak,
                                         bd + (uint64_t)(k * 128 + s * tap_step), idesc, acc_in);
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
        const int S = prm.S;
        for (int u = blockIdx.x; u < prm.units; u += gridDim.x, ++local) {
            int slice, kt, r, ct;
            unit_decode(prm, u, slice, kt, r, ct);
            const int acc = prm.nacc == 2 ? (local & 1) : 0;
            const uint32_t aph = (uint32_t)((prm.nacc == 2 ? local >> 1 : local) & 1);
            if (!ptx::mbar_wait(&tfull[acc], aph, lim, abort_flag)) {
                fail();
                break;
            }
            ptx::tc_fence_after();
            const int k0 = kt * KT + quarter * 32;
            const int nchunks = S * (BN / 32);
            for (int ch = 0; ch < nchunks; ++ch) {
                const int s = ch / (BN / 32), j = ch - s * (BN / 32);
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(acc * prm.acc_cols + ch * 32),
                                        v);
                ptx::tmem_ld_wait();
                if (ch == nchunks - 1) {
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                }
                if (k0 >= prm.K) continue;
                uint8_t *bp = sbuf + ebuf * 4096;
                if (lane == 0) ptx::bulk_wait_read<1>();
                __syncwarp();
                uint8_t *dst = bp + lane * 128;  // row = output channel k0 + lane
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4 *>(dst + ((c ^ (lane & 7)) << 4)) =
                        make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    ptx::tma_store_4d(&prm.tmW, bp, ct * BN + j * 32, r * S + s, k0, slice);
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
    if (warp == 1) ptx::tmem_dealloc(tmem_base, (uint32_t)prm.tcols);
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Band geometry: the input-channel tile, the row width Wx, and the rows per
// band TR that minimise the padded MMA work per image (plus a fixed cost per
// band) with at least two pipeline stages in shared memory. Returns false when
// the layer does not fit this kernel.
bool plan(const Dims &d, Plan *pl) {
    if (d.layout != GBCONV_NHWC || d.in_dtype != GBCONV_BF16 || d.G != 1) return false;
    if (d.u != 1 || d.v != 1 || d.C % 64 || d.K % 8) return false;
    if (d.R * d.S < 2 || d.P < 1 || d.Q < 1) return false;
    if (d.M() >= (1ll << 31)) return false;
    const int bn = (d.C % 128 == 0 && d.S * 128 <= 512) ? 128 : 64;
    if (d.S * bn > 512) return false;  // the S accumulators in TMEM
    const int wx = d.Q + std::max(0, (d.S - 1) * d.dw - d.pw);
    if (wx > 256) return false;  // a TMA box dimension
    // TMA coordinates of the x box start (int32)
    if ((long long)d.ph + (long long)(d.R - 1) * d.dh > (1ll << 30) || d.pw > (1 << 20)) return false;
    int best_cost = -1;
    Plan bestp{};
    for (int tr = 1; tr <= std::min(d.P, 256); ++tr) {
        const int vrow = tr * wx;
        const int jpad = round_up(vrow, 16);
        const int xrows = round_up(jpad + (d.S - 1) * d.dw, 8);
        const int a_blk = jpad * 128, b_blk = xrows * 128;
        const int stage = 2 * a_blk + (bn / 64) * b_blk;
        const int stages = std::min(MAX_STAGES, (SMEM_LIMIT - SMEM_ALIGN - EPI_TOTAL - BAR_BYTES) / stage);
        if (stages < 2) break;  // larger bands only grow
        const int bpi = (d.P + tr - 1) / tr;
        const int cost = bpi * (jpad + 32);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            bestp.bn = bn;
            bestp.wx = wx;
            bestp.tr = tr;
            bestp.jpad = jpad;
            bestp.xrows = xrows;
            bestp.a_blk = a_blk;
            bestp.b_blk = b_blk;
            bestp.stages = stages;
            bestp.bpi = bpi;
        }
    }
    if (best_cost < 0) return false;
    bestp.acc_cols = d.S * bn;
    bestp.nacc = 2 * bestp.acc_cols <= 512 ? 2 : 1;
    const int need = bestp.nacc * bestp.acc_cols;
    int tc = 32;
    while (tc < need) tc *= 2;
    bestp.tcols = tc;
    *pl = bestp;
    return true;
}

size_t smem_bytes(const Plan &pl) {
    return (size_t)SMEM_ALIGN + (size_t)pl.stages * (2 * pl.a_blk + (pl.bn / 64) * pl.b_blk) +
           EPI_TOTAL + BAR_BYTES;
}

template <int BN>
gbconv_status_t launch(const WsParams &prm, size_t smem, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_wgrad_shift_kernel<BN>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    });
    if (attr_err != cudaSuccess) return cuda_status(attr_err);
    return cuda_status(launch_pdl(tc_wgrad_shift_kernel<BN>, dim3(grid), dim3(NTHREADS), smem, st, prm));
}

}  // namespace

bool tc_wgrad_shift_supported(const Dims &d) {
    Plan pl;
    return plan(d, &pl);
}

long long tc_wgrad_shift_bands(const Dims &d) {
    Plan pl;
    if (!plan(d, &pl)) return 0;
    return (long long)d.N * pl.bpi;
}

int tc_wgrad_shift_default_slices(const Dims &d) {
    Plan pl;
    if (!plan(d, &pl)) return 1;
    const long long per_slice = (long long)((d.K + KT - 1) / KT) * d.R * (d.C / pl.bn);
    const long long nbands = (long long)d.N * pl.bpi;
    long long s = per_slice >= SMS_FOR_DEFAULTS ? 1 : SMS_FOR_DEFAULTS / per_slice;
    s = std::min<long long>(s, std::max<long long>(nbands, 1));
    s = std::min<long long>(s, 256);
    return (int)std::max<long long>(s, 1);
}

gbconv_status_t launch_tc_wgrad_shift_partials(const Dims &d, int slices, const void *x, const void *g,
                                               float *ws, cudaStream_t st) {
    Plan pl;
    if (!plan(d, &pl)) return GBCONV_ERR_UNSUPPORTED;
    const long long nbands = (long long)d.N * pl.bpi;
    if (nbands >= (1ll << 31)) return GBCONV_ERR_UNSUPPORTED;
    if (slices < 1 || slices > nbands) return GBCONV_ERR_INVALID_ARG;  // every slice needs a band
    WsParams prm;
    memset(&prm, 0, sizeof(prm));
    // dy as [N][P][Q][K]; a band box is 64 channels x Wx positions x TR rows
    uint64_t gdims[4] = {(uint64_t)d.K, (uint64_t)d.Q, (uint64_t)d.P, (uint64_t)d.N};
    uint64_t gstr[3] = {(uint64_t)d.K * 2, (uint64_t)d.Q * d.K * 2, (uint64_t)d.P * d.Q * d.K * 2};
    uint32_t box[4] = {64, (uint32_t)pl.wx, (uint32_t)pl.tr, 1};
    gbconv_status_t s = encode_tiled(&prm.tmG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, g, gdims, gstr,
                                     box, CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    uint64_t xdims[4] = {(uint64_t)d.C, (uint64_t)d.W, (uint64_t)d.H, (uint64_t)d.N};
    uint64_t xstr[3] = {(uint64_t)d.C * 2, (uint64_t)d.W * d.C * 2, (uint64_t)d.H * d.W * d.C * 2};
    s = encode_tiled(&prm.tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, x, xdims, xstr, box,
                     CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    // partials [slices][K][R*S][C], FP32, stored in 32 x 32 chunks
    const int RS = d.R * d.S;
    uint64_t wdims[4] = {(uint64_t)d.C, (uint64_t)RS, (uint64_t)d.K, (uint64_t)slices};
    uint64_t wstr[3] = {(uint64_t)d.C * 4, (uint64_t)RS * d.C * 4, (uint64_t)d.K * RS * d.C * 4};
    uint32_t wbox[4] = {32, 1, 32, 1};
    s = encode_tiled(&prm.tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ws, wdims, wstr, wbox,
                     CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != GBCONV_OK) return s;
    prm.K = d.K;
    prm.S = d.S;
    prm.dw = d.dw;
    prm.ph = d.ph;
    prm.pw = d.pw;
    prm.dh = d.dh;
    prm.tr = pl.tr;
    prm.bpi = pl.bpi;
    prm.nbands = (int)nbands;
    prm.ksteps = pl.jpad / 16;
    prm.valid_rows = pl.tr * pl.wx;
    prm.xrows = pl.xrows;
    prm.jpad = pl.jpad;
    prm.a_blk = pl.a_blk;
    prm.b_blk = pl.b_blk;
    prm.stages = pl.stages;
    prm.acc_cols = pl.acc_cols;
    prm.nacc = pl.nacc;
    prm.tcols = pl.tcols;
    prm.nprod = std::min(NPROD, pl.stages);
    prm.k_tiles = (d.K + KT - 1) / KT;
    prm.c_tiles = d.C / pl.bn;
    prm.R = d.R;
    prm.slices = slices;
    const long long units = (long long)slices * prm.k_tiles * d.R * prm.c_tiles;
    if (units >= (1ll << 31)) return GBCONV_ERR_UNSUPPORTED;
    prm.units = (int)units;
    prm.guard = make_guard();
    if (!prm.guard.err) return GBCONV_ERR_CUDA;
    const int grid = (int)std::min<long long>(units, sm_count());
    const size_t smem = smem_bytes(pl);
    if (pl.bn == 128) return launch<128>(prm, smem, grid, st);
    return launch<64>(prm, smem, grid, st);
}

}  // namespace gbc
