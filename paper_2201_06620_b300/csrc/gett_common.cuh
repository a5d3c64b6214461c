// Device-side pieces shared by the GETT kernel files.
#pragma once

#include "internal.h"

namespace rosnet {

struct GroupArgs {
    const GettDesc *descs;  // device array, or NULL to use `single`
    int ndesc;
    GettDesc single;
};

// Locate this CTA's problem (the last one whose tile_begin <= blockIdx.x).
__device__ __forceinline__ void load_desc(const GroupArgs &g, GettDesc &sd) {
    if (g.descs == nullptr) {
        sd = g.single;
        return;
    }
    const int64_t bid = blockIdx.x;
    int lo = 0, hi = g.ndesc - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g.descs[mid].tile_begin <= bid) lo = mid;
        else hi = mid - 1;
    }
    sd = g.descs[lo];
}


// Device status word: kernels set a nonzero code when a bounded wait gives up
// (see rosnet_sync).
enum : int32_t { kDevErrNone = 0, kDevErrTimeout = 1 };

}  // namespace rosnet
