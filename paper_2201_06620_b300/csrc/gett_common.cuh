// Device-side pieces shared by the GETT kernel files.
#pragma once

#include <cstring>

#include "internal.h"

namespace rosnet {

struct GroupArgs {
    const GettDesc *descs;  // device array, or NULL to use `single`
    int ndesc;
    GettDesc single;
};

// Locate this CTA's problem (the last one whose tile_begin <= blockIdx.x)
// and copy its descriptor to shared memory.  Called by all 32 lanes of one
// warp: each round the lanes read 32 tile_begin values spread over the
// remaining range at once, so a launch of n problems costs ceil(log32 n)
// dependent loads instead of log2 n; the lanes then copy the descriptor
// word by word.
__device__ __forceinline__ void load_desc(const GroupArgs &g, GettDesc &sd) {
    static_assert(sizeof(GettDesc) % 8 == 0, "descriptor is copied in 8-byte words");
    constexpr int kWords = (int)(sizeof(GettDesc) / 8);
    const int lane = threadIdx.x & 31;
    const GettDesc *src = &g.single;
    if (g.descs != nullptr) {
        const int64_t bid = blockIdx.x;
        int lo = 0, n = g.ndesc;   // answer in [lo, lo + n); descs[lo].tile_begin <= bid
        while (n > 1) {
            const int step = (n + 31) >> 5;
            const int idx = lo + lane * step;
            const bool le = idx < lo + n && __ldg(&g.descs[idx].tile_begin) <= bid;
            const unsigned mask = __ballot_sync(0xffffffffu, le);   // bit 0 always set
            const int nlo = lo + (31 - __clz((int)mask)) * step;
            n = min(step, lo + n - nlo);
            lo = nlo;
        }
        src = g.descs + lo;
    }
    const int64_t *s = reinterpret_cast<const int64_t *>(src);
    int64_t *d = reinterpret_cast<int64_t *>(&sd);
    for (int w = lane; w < kWords; w += 32) d[w] = s[w];
}


// Programmatic dependent launch.  Kernels launched with the programmatic
// stream-serialization attribute may start while the previous kernel in the
// stream is still running: grid_dep_launch() lets the next kernel begin its
// prologue, and grid_dep_wait() blocks until the previous kernel has finished
// and its writes are visible.  Before grid_dep_wait() a kernel reads only its
// descriptor and offset tables, and every CTA calls it before touching
// operands or results and before it exits, so the completion of a grid still
// implies the completion of all earlier grids.  Without the attribute both
// are no-ops.
//
// The prologue's reads are safe only if the descriptor and tables were
// complete before the previous kernel in the stream started.  Tables uploaded
// by a copy are; tables written by a kernel (build_table_kernel) are not when
// that kernel is the one immediately before: the launch that follows a table
// build therefore passes pdl = false and starts only after the build has
// completed and its writes are visible.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch a kernel, with programmatic stream serialization when pdl is set (its
// prologue then overlaps the end of the previous kernel in the stream; the
// kernel calls grid_dep_wait() before it touches operands, workspaces or
// results), else in plain stream order.
template <typename Kern, typename... Args>
inline void launch_pdl(Kern kern, dim3 grid, unsigned threads, size_t smem, cudaStream_t s, bool pdl,
                       const Args &...args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    RN_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

// Device status word: kernels set a nonzero code when a bounded wait gives up
// (see rosnet_sync).
enum : int32_t { kDevErrNone = 0, kDevErrTimeout = 1 };

}  // namespace rosnet
