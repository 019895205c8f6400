// epilogue.cuh -- shared epilogue of the tensor-core forward kernels: one
// 32 x 32 accumulator chunk from TMEM registers to y through a swizzled
// shared-memory buffer and a TMA tensor store.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"
#include "ptx.cuh"

namespace gbc {

// Epilogue shape per tile width: 256-column tiles carry the most output per
// MMA, so they get 16 epilogue warps (four per TMEM lane quarter) to hide the
// per-chunk latency chain; narrower tiles get 8. Either way the warps share 64
// KB of staging: NBUF 2 KB BF16 chunk buffers per warp (NBUF-1 TMA stores may
// still be reading while one is filled), or NBUF/2 4 KB FP32 ones.
constexpr int EPI_TOTAL_BYTES = 65536;
template <int BN>
struct EpiShape {
    static constexpr int warps = BN >= 256 ? 16 : 8;
    static constexpr int threads = 64 + 32 * warps;  // + producer and MMA warps
    static constexpr int warp_bytes = EPI_TOTAL_BYTES / warps;
    static constexpr int nbuf = warp_bytes / 2048;   // 2 or 4
};

// What the epilogue needs to know about the output.
struct EpiArgs {
    int K;                 // output channels (columns >= K are never stored)
    int relu, out_f32;
    const float *bias;     // [K] or null
    const float *w_scale;  // [K] FP8 per-channel scales (FP8 only)
    const float *alpha;    // [K] fused per-channel scale (folded batch norm) or null
    const void *z;         // fused residual, y's shape and dtype (may be y) or null
    long long M;           // rows of y as [M][K] (2-D stores)
    int Q;                 // row length of y as [N*P][Q][K] (3-D stores)
};

__device__ __forceinline__ void store_chunk(const CUtensorMap *map, const void *src, int c0, int c1,
                                            int c2) {
    if (c2 < 0)
        ptx::tma_store_2d(map, src, c0, c1);
    else
        ptx::tma_store_3d(map, src, c0, c1, c2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a -> low half
    return *reinterpret_cast<uint32_t *>(&h);
}

// Epilogue of one 32-row x 32-column accumulator chunk held by a warp (lane =
// row): scale, bias, ReLU, convert, stage in shared memory in the layout the
// TMA store's swizzle expects, and store the chunk with one TMA instruction
// at coordinates (col0, c1) of a 2-D map, or (col0, c1, c2) of a 3-D map when
// c2 >= 0.
//   BF16 output: 32 rows x 64 B, 64-byte swizzle (16-B unit c of row r sits at
//                unit c ^ ((r >> 1) & 3)), NBUF 2 KB buffers used in turn;
//   FP32 output: 32 rows x 128 B, 128-byte swizzle (unit c ^ (r & 7)), NBUF/2
//                4 KB buffers used in turn.
// Residual values of this lane's row, columns col0 .. col0+31 (0 outside y).
__device__ __forceinline__ void load_residual(const EpiArgs &pa, int col0, int c1, int c2,
                                              int lane, float (&zr)[32]) {
    long long row;
    bool valid;
    if (c2 < 0) {
        row = (long long)c1 + lane;
        valid = row < pa.M;
    } else {
        row = (long long)c2 * pa.Q + c1 + lane;
        valid = c1 + lane < pa.Q;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {  // 8 channels per 16-byte (BF16) or 32-byte (FP32) group
        const int c = col0 + 8 * g;
        const bool ok = valid && c < pa.K;  // K is a multiple of 8
        if (pa.out_f32) {
            const float4 *p = reinterpret_cast<const float4 *>(
                static_cast<const float *>(pa.z) + (ok ? row * pa.K + c : 0));
            const float4 a = ok ? p[0] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 b = ok ? p[1] : make_float4(0.f, 0.f, 0.f, 0.f);
            zr[8 * g + 0] = a.x; zr[8 * g + 1] = a.y; zr[8 * g + 2] = a.z; zr[8 * g + 3] = a.w;
            zr[8 * g + 4] = b.x; zr[8 * g + 5] = b.y; zr[8 * g + 6] = b.z; zr[8 * g + 7] = b.w;
        } else {
            const uint4 u = ok ? *reinterpret_cast<const uint4 *>(
                                     static_cast<const __nv_bfloat16 *>(pa.z) + row * pa.K + c)
                               : make_uint4(0, 0, 0, 0);
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                zr[8 * g + 2 * i] = f.x;
                zr[8 * g + 2 * i + 1] = f.y;
            }
        }
    }
}

// FUSED instantiations also apply the per-channel scale and the residual
// (EpiArgs::alpha, EpiArgs::z); the others ignore both fields.
// Asks L2 for the residual values this lane will add for a chunk at columns
// col0 .. col0+31 (the same rows as load_residual), ahead of the accumulator.
__device__ __forceinline__ void prefetch_residual(const EpiArgs &pa, int col0, int c1, int c2,
                                                  int lane) {
    long long row;
    bool valid;
    if (c2 < 0) {
        row = (long long)c1 + lane;
        valid = row < pa.M;
    } else {
        row = (long long)c2 * pa.Q + c1 + lane;
        valid = c1 + lane < pa.Q;
    }
    if (!valid || col0 >= pa.K) return;
    const int eb = pa.out_f32 ? 4 : 2;
    const char *p = static_cast<const char *>(pa.z) + (row * pa.K + col0) * eb;
    ptx::prefetch_l2(p);
    ptx::prefetch_l2(p + 32 * eb - 1);  // the chunk's last byte (may be the next line)
}

// Fused epilogue of one BF16-output chunk whose residual tile was brought into
// the 2 KB staging buffer `b` by a TMA load with the store's own map shape
// (32 rows x 64 B, 64-byte swizzle): each lane reads its row's 32 residual
// values from the buffer, adds them (after scale and bias), writes the
// results over them in place and the buffer is stored with one TMA store.
// The caller has waited for the load.
template <bool FP8>
__device__ __forceinline__ void epilogue_chunk_zsmem(const uint32_t (&v)[32], const EpiArgs &pa,
                                                     const CUtensorMap *tmY, float xs, int col0,
                                                     int c1, int c2, int lane, uint8_t *b) {
    float scl = 1.f, bl = 0.f, al = 1.f;
    const int mycol = col0 + lane;
    if (mycol < pa.K) {
        if (FP8) scl = xs * __ldg(pa.w_scale + mycol);
        if (pa.bias) bl = __ldg(pa.bias + mycol);
        if (pa.alpha) al = __ldg(pa.alpha + mycol);
    }
    uint8_t *row = b + lane * 64;
    float f[32];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint4 u = *reinterpret_cast<const uint4 *>(row + ((c ^ ((lane >> 1) & 3)) << 4));
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 z2 = __bfloat1622float2(h[i]);
            f[8 * c + 2 * i] = z2.x;
            f[8 * c + 2 * i + 1] = z2.y;
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float a = __uint_as_float(v[i]);
        if (FP8) a = a * __shfl_sync(0xffffffffu, scl, i);
        if (pa.alpha) a = a * __shfl_sync(0xffffffffu, al, i);
        if (pa.bias) a = a + __shfl_sync(0xffffffffu, bl, i);
        a = a + f[i];
        if (pa.relu) a = fmaxf(a, 0.f);
        f[i] = a;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4 *>(row + ((c ^ ((lane >> 1) & 3)) << 4)) =
            make_uint4(pack_bf16(f[8 * c], f[8 * c + 1]), pack_bf16(f[8 * c + 2], f[8 * c + 3]),
                       pack_bf16(f[8 * c + 4], f[8 * c + 5]), pack_bf16(f[8 * c + 6], f[8 * c + 7]));
    ptx::fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
        store_chunk(tmY, b, col0, c1, c2);
        ptx::bulk_commit();
    }
}

template <bool FP8, int NBUF, bool FUSED = false>
__device__ __forceinline__ void epilogue_chunk(const uint32_t (&v)[32], const EpiArgs &pa,
                                               const CUtensorMap *tmY, float xs, int col0,
                                               int c1, int c2, int lane, uint8_t *sbuf, int &ebuf) {
    float scl = 1.f, bl = 0.f, al = 1.f;
    const int mycol = col0 + lane;
    if (mycol < pa.K) {
        if (FP8) scl = xs * __ldg(pa.w_scale + mycol);
        if (pa.bias) bl = __ldg(pa.bias + mycol);
        if (FUSED && pa.alpha) al = __ldg(pa.alpha + mycol);
    }
    float zr[FUSED ? 32 : 1];
    if constexpr (FUSED) {
        if (pa.z) load_residual(pa, col0, c1, c2, lane, zr);
    }
    float f[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float a = __uint_as_float(v[i]);
        if (FP8) a = a * __shfl_sync(0xffffffffu, scl, i);
        if constexpr (FUSED) {
            if (pa.alpha) a = a * __shfl_sync(0xffffffffu, al, i);
        }
        if (pa.bias) a = a + __shfl_sync(0xffffffffu, bl, i);
        if constexpr (FUSED) {
            if (pa.z) a = a + zr[i];
        }
        if (pa.relu) a = fmaxf(a, 0.f);
        f[i] = a;
    }
    if (pa.out_f32) {
        uint8_t *b = sbuf + (ebuf % (NBUF / 2)) * 4096;
        if (lane == 0) ptx::bulk_wait_read<NBUF / 2 - 1>();
        __syncwarp();
        uint8_t *dst = b + lane * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4 *>(dst + ((c ^ (lane & 7)) << 4)) =
                make_uint4(__float_as_uint(f[4 * c]), __float_as_uint(f[4 * c + 1]),
                           __float_as_uint(f[4 * c + 2]), __float_as_uint(f[4 * c + 3]));
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            store_chunk(tmY, b, col0, c1, c2);
            ptx::bulk_commit();
        }
        ebuf = (ebuf + 1) % (NBUF / 2);
    } else {
        uint8_t *b = sbuf + ebuf * 2048;
        if (lane == 0) ptx::bulk_wait_read<NBUF - 1>();
        __syncwarp();
        uint8_t *dst = b + lane * 64;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(dst + ((c ^ ((lane >> 1) & 3)) << 4)) =
                make_uint4(pack_bf16(f[8 * c], f[8 * c + 1]), pack_bf16(f[8 * c + 2], f[8 * c + 3]),
                           pack_bf16(f[8 * c + 4], f[8 * c + 5]),
                           pack_bf16(f[8 * c + 6], f[8 * c + 7]));
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            store_chunk(tmY, b, col0, c1, c2);
            ptx::bulk_commit();
        }
        ebuf = (ebuf + 1) % NBUF;
    }
}


}  // namespace gbc
