// Kernel launches of the library: one helper, so that every kernel can take part in programmatic
// dependent launch inside the captured iteration graphs.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace kcm {

// Launches kernel<<<grid, block, smem, s>>>(args...). With pdl, the launch allows programmatic stream
// serialization: the kernel's blocks may be scheduled while the previous kernel of the stream is still
// running (it lets them go once all its blocks have started), and the kernel's first statement,
// grid_dep_sync (griddepcontrol.wait), holds every thread until that kernel has completed and its
// memory operations are visible. So only the launch latency overlaps; no data moves early.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int pdl,
                     Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface at the next check
}

}  // namespace kcm
