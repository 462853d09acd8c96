// Programmatic dependent launch (sm_90 and later): a kernel launched with programmatic stream serialization
// may be scheduled while the kernel before it on the stream is still finishing; it waits for that kernel's
// completion and memory (griddepcontrol.wait) before it touches global memory.  Chains of small latency-bound
// kernels then overlap each launch with the tail of the kernel before it.
//
// Every kernel launched through launch_k calls pdl_wait() before its first global memory access; launched
// without the attribute (SCBB_PDL=0, or a stream op other than a kernel before it) the wait returns at once.
// pdl_trigger() lets the next kernel be scheduled before this one ends (it still waits for its completion).
#pragma once

#include <stdlib.h>

#include <utility>

namespace scbb {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

inline bool pdl_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SCBB_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// kernel<<<grid, block, smem, st>>>(args...), with programmatic stream serialization unless disabled
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
    if (!pdl_enabled()) {
        kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
        return cudaPeekAtLastError();
    }
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

}  // namespace scbb
