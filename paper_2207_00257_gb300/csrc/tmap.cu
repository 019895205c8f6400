// tmap.cu -- TMA tensor-map encoding. The driver's cuTensorMapEncode* entry
// points are fetched once through the runtime (no link against libcuda).
#include <mutex>

#include "internal.h"

namespace gbc {
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
using EncodeIm2colFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const int *,
                                    const int *, cuuint32_t, cuuint32_t, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn g_tiled = nullptr;
EncodeIm2colFn g_im2col = nullptr;
std::once_flag g_once;

void load_entry_points() {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_tiled = reinterpret_cast<EncodeTiledFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_im2col = reinterpret_cast<EncodeIm2colFn>(p);
}

}  // namespace

// Im2col map over an NHWC activation x[N][H][W][C]. The bounding box runs
// from (-pw, -ph) to (W-1 + pw - dw(S-1), H-1 + ph - dh(R-1)): the positions of
// the filter's top-left tap, visited with the convolution strides (v, u), so
// that the walk over one column enumerates output pixels (n, p, q) in order,
// crossing rows and images. Taps out of the image read as zeros.
gbconv_status_t encode_im2col_act(CUtensorMap *m, const Dims &d, const void *x, int elem_bytes,
                                  int channels_per_pixel, int pixels_per_column) {
    std::call_once(g_once, load_entry_points);
    if (!g_im2col) return GBCONV_ERR_CUDA;
    if (reinterpret_cast<uintptr_t>(x) % 16) return GBCONV_ERR_ALIGNMENT;
    const cuuint64_t ldc = (cuuint64_t)d.xstride();  // channels between pixels
    cuuint64_t dims[4] = {(cuuint64_t)d.C, (cuuint64_t)d.W, (cuuint64_t)d.H, (cuuint64_t)d.N};
    cuuint64_t strides[3] = {ldc * elem_bytes, (cuuint64_t)d.W * ldc * elem_bytes,
                             (cuuint64_t)d.H * d.W * ldc * elem_bytes};
    int lower[2] = {-d.pw, -d.ph};
    int upper[2] = {d.pw - d.dw * (d.S - 1), d.ph - d.dh * (d.R - 1)};
    cuuint32_t estr[4] = {1, (cuuint32_t)d.v, (cuuint32_t)d.u, 1};
    CUresult r = g_im2col(m, elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          4, const_cast<void *>(x), dims, strides, lower, upper,
                          (cuuint32_t)channels_per_pixel, (cuuint32_t)pixels_per_column, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GBCONV_OK : GBCONV_ERR_CUDA;
}

gbconv_status_t encode_tiled(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *ptr,
                             const uint64_t *dims, const uint64_t *strides_bytes,
                             const uint32_t *box, CUtensorMapSwizzle swz,
                             const uint32_t *elem_strides) {
    std::call_once(g_once, load_entry_points);
    if (!g_tiled) return GBCONV_ERR_CUDA;
    if (reinterpret_cast<uintptr_t>(ptr) % 16) return GBCONV_ERR_ALIGNMENT;
    cuuint64_t gd[5];
    cuuint64_t gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = elem_strides ? elem_strides[i] : 1;
        if (i + 1 < rank) {
            gs[i] = strides_bytes[i];
            if (gs[i] % 16) return GBCONV_ERR_ALIGNMENT;
        }
    }
    CUresult r = g_tiled(m, dt, (cuuint32_t)rank, const_cast<void *>(ptr), gd, gs, bx, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GBCONV_OK : GBCONV_ERR_CUDA;
}

}  // namespace gbc
