// launch.cuh -- every kernel of the library is launched through launch_pdl:
// cudaLaunchKernelEx with programmatic stream serialization, so that a
// kernel's launch and prologue overlap the tail of the kernel before it on
// the stream. Kernels call ptx::griddep_wait() before touching global memory,
// which keeps the stream's ordering semantics exact.
#pragma once

#include <cuda_runtime.h>

namespace gbc {

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace gbc
