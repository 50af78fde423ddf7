// mg_launch.cuh -- programmatic dependent launch (PTX ISA: griddepcontrol;
// CUDA launch attribute programmaticStreamSerialization).
//
// A kernel launched with the attribute may be scheduled onto the SMs while the
// kernel before it in the stream (or the graph node before it, when captured)
// is still running.  Every kernel of this library begins with dep_entry() (the
// staged one-pass sweep with dep_wait(), and dep_release() at its end):
//   griddepcontrol.wait              holds the block until the preceding grid
//                                    has completed and its memory operations
//                                    are visible (returns at once when the
//                                    kernel was launched without the attribute);
//   griddepcontrol.launch_dependents then allows the next kernel to be scheduled
//                                    once every block of this grid has passed
//                                    here (or exited).
// Waiting first keeps the ordering of a plain stream for every access, reads and
// writes alike; what the attribute removes is the launch latency between two
// dependent kernels: the next grid's blocks are resident and waiting when this
// one retires.  Only the next grid is allowed early, and only after every block
// of this one is running, so a waiting grid never holds resources that this
// one still needs.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace gbmg {

__device__ __forceinline__ void dep_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The two halves of dep_entry for a kernel whose SMs should not host the next
// grid's waiting blocks while it runs (an issue-bound kernel that leaves room
// for them): wait at entry, allow the next grid only when the block is done.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches made by this host thread carry the attribute while a DepScope with
// on = 1 is alive (plan execution and graph capture); elsewhere (autotuner
// timing, per-launch event profiling, single-kernel entry points) they are
// plain launches.
extern thread_local int tl_dep_launch;

struct DepScope {
    int old;
    explicit DepScope(int on) : old(tl_dep_launch) { tl_dep_launch = on; }
    ~DepScope() { tl_dep_launch = old; }
    DepScope(const DepScope &) = delete;
    DepScope &operator=(const DepScope &) = delete;
};

// kernel<<<grid, block, smem, s>>>(args...), with the attribute when enabled.
// Errors are left in the runtime's last-error state, as for <<< >>>.
template <typename... P, typename... A>
inline void launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = s;
    c.attrs = at;
    c.numAttrs = tl_dep_launch ? 1u : 0u;
    cudaLaunchKernelEx(&c, kernel, std::forward<A>(args)...);
}

// Process default for plans: on unless the environment sets MG_DEP_LAUNCH=0.
int dep_launch_default();

}  // namespace gbmg
