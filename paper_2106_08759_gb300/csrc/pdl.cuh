// pdl.cuh -- programmatic dependent launch (internal).
//
// The kernels of one stream's chain (sampling, the tree levels, the root
// inversions, h and the encodings, the hash, the fix-up) may be launched
// with programmatic stream serialization: the next kernel's CTAs are then
// scheduled while the previous kernel's last wave still runs, and wait in
// hardware (griddepcontrol.wait) until that kernel has completed and its
// writes are visible, which hides the launch gap between dependent kernels.
//
// Every kernel that may be launched this way begins with pdl_enter(): the
// wait comes before any memory access and before any early return, so a
// kernel's completion always implies its predecessor's (a CTA that left
// before waiting could let the kernel after it run ahead of the one before
// it).  Only then does it allow its own dependents to launch.  Without the
// launch attribute both instructions are no-ops.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace snt {

__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A kernel of the chain starts when every CTA of its predecessor has passed
// pdl_enter, that is, when the kernel before that has completed: so a kernel
// may read, before its own pdl_enter, data written by kernels two or more
// launches back in its own stream, never data of its immediate predecessor,
// and never data of another stream joined by an event (captured in a graph,
// that edge too may become programmatic); it may write nothing there.  Each
// CTA still calls pdl_enter before it exits.

// Whether launches on this host thread use the attribute: set for the
// duration of one library call from its context's option (PdlScope).
inline thread_local bool tl_pdl = false;

struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(tl_pdl) { tl_pdl = on; }
    ~PdlScope() { tl_pdl = prev; }
    PdlScope(const PdlScope &) = delete;
    PdlScope &operator=(const PdlScope &) = delete;
};

// kernel<<<grid, block, smem, st>>>(args...), with programmatic stream
// serialization when this thread's calls enable it.  The kernel must begin
// with pdl_enter().
template <typename... KP, typename... A>
cudaError_t launch_k(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     A &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = tl_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

}  // namespace snt

// SNT_LAUNCH(kernel, grid, block, smem, stream, args...): launch_k, returning
// its error from the enclosing function.
#define SNT_LAUNCH(...)                                             \
    do {                                                            \
        const cudaError_t snt_le_ = ::snt::launch_k(__VA_ARGS__);   \
        if (snt_le_ != cudaSuccess) return snt_le_;                 \
    } while (0)
