// launch.cuh -- kernel launches with programmatic dependent launch.
//
// Every kernel of the step begins with pdl_enter(): it waits until the kernel
// before it in the stream has completed and its writes are visible
// (griddepcontrol.wait), then allows the next kernel to be launched
// (griddepcontrol.launch_dependents), so that the next kernel's blocks are
// scheduled while this one runs and start the moment it ends instead of
// after a launch latency.  Because each kernel waits for its predecessor
// before anything else -- returning included -- completion is transitive
// along the stream, and no kernel reads a result before it is complete.
// Launched without the attribute (or by a plain <<< >>>), both instructions
// return at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

// 0: plain stream-ordered launches (the kernels' griddepcontrol
// instructions then return at once)
#ifndef DEM_PDL
#define DEM_PDL 1
#endif

namespace dem {

// Whether launch_pdl sets the attribute, chosen by the world before it
// captures its step (per host thread: a world is used by one thread at a
// time).  Measured per step with and without: 1,000 spheres 82 -> 76 us, but
// 2e4 spheres 224 -> 231 us and 1e5 spheres 2.872 -> 2.891 ms, so worlds
// above 8,192 spheres launch plainly.
inline thread_local bool tl_pdl = true;
constexpr int64_t kPdlMaxSpheres = 8192;

__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kernel<<<grid, block, smem, st>>>(args...) with the programmatic
// stream-serialisation attribute; the status is left for cudaGetLastError.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (DEM_PDL && tl_pdl) ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace dem
