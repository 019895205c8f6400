// tc_wgrad.cu -- tensor-core weight gradient (placeholder until the tcgen05
// kernel lands: every problem goes to the CUDA-core partial-sum kernel).
#include "internal.h"

namespace gbc {

bool tc_wgrad_supported(const Dims &) { return false; }

TcConfig tc_wgrad_default_config(const Dims &) { return TcConfig{0, 0, 1, 0}; }

gbconv_status_t launch_tc_wgrad_partials(const Dims &, const TcConfig &, const void *,
                                         const void *, float *, cudaStream_t) {
    return GBCONV_ERR_UNSUPPORTED;
}

}  // namespace gbc
