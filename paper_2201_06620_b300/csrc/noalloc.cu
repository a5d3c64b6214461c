// rosnet_tensordot_noalloc: the pairwise tensordot for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they contract: code that runs inside a framework that owns all device
// memory and forbids foreign allocations, real-time or embedded callers with
// a fixed, pre-committed memory budget, and callers on a path where an
// allocation could block or fail unpredictably.  They pass inputs and an
// already created output tensor; the scratch the kernels need (offset tables,
// split-K partial sums, packed operands) lives in one file-scope device array
// of fixed size instead of coming from an allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace rosnet {

void check_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axes_a,
                     const int *axes_b, int *axa, int *axb, int &rc, int64_t *shc, int64_t *blc);
int check_precision(const rosnet_opts *opts, int dtype);
size_t tensordot_into_ws(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axa,
                         const int *axb, rosnet_btensor C, int precision, int reduce_mode, void *ws,
                         size_t ws_bytes, cudaStream_t s);

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ROSNET_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached for the life of the
// process (a device reset would invalidate it; the header says so).
void *scratch_on_current_device() {
    int dev = 0;
    RN_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        RN_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

// Bytes [lo, hi) that a tensor's two planes can touch: from its data pointer
// to one past the last element of its imaginary plane.
void storage_range(rosnet_btensor t, uintptr_t *lo, uintptr_t *hi) {
    int64_t last = 0;   // largest element offset within a plane
    for (int i = 0; i < t->lay.rank; ++i) {
        const int64_t b = t->lay.block[i], g = t->lay.shape[i] / b;
        last += (g - 1) * t->lay.gstride[i] + (b - 1) * t->lay.lstride[i];
    }
    *lo = (uintptr_t)t->data;
    *hi = *lo + (uintptr_t)((t->pstride + last + 1) * (int64_t)t->elsize);
}

bool storage_overlaps(rosnet_btensor x, rosnet_btensor y) {
    uintptr_t xl, xh, yl, yh;
    storage_range(x, &xl, &xh);
    storage_range(y, &yl, &yh);
    return xl < yh && yl < xh;
}

}  // namespace
}  // namespace rosnet

using namespace rosnet;

extern "C" rosnet_status rosnet_tensordot_noalloc(rosnet_btensor A, rosnet_btensor B, int naxes,
                                                  const int *axes_a, const int *axes_b,
                                                  rosnet_btensor C, const rosnet_opts *opts,
                                                  void *stream) {
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    if (!C) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL output tensor");
    int axa[kMaxRank], axb[kMaxRank], rc = 0;
    int64_t shc[kMaxRank], blc[kMaxRank];
    check_tensordot(A, B, naxes, axes_a, axes_b, axa, axb, rc, shc, blc);
    if (C->lay.numel > 0 && (storage_overlaps(C, A) || storage_overlaps(C, B)))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "the output's storage overlaps an operand's");
    if (C->dtype != A->dtype) RN_FAIL(ROSNET_ERR_DTYPE, "output dtype differs from the operands'");
    if (C->lay.rank != rc) RN_FAIL(ROSNET_ERR_SHAPE, "output rank does not match the result");
    for (int i = 0; i < rc; ++i) {
        if (C->lay.shape[i] != shc[i]) RN_FAIL(ROSNET_ERR_SHAPE, "output shape does not match the result");
        if (C->lay.block[i] != blc[i])
            RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "output block shape does not match the result");
    }
    const int prec = check_precision(opts, A->dtype);
    const int red = check_reduce(opts);
    if (opts && (opts->flags & ROSNET_OPT_AUTOTUNE))
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "autotuning times candidate kernels in buffers of their own; "
                                        "rosnet_tensordot_noalloc allocates nothing");
    void *ws = scratch_on_current_device();
    const size_t need = tensordot_into_ws(A, B, naxes, axa, axb, C, prec, red, ws,
                                          ROSNET_NOALLOC_SCRATCH_BYTES, s);
    if (need > (size_t)ROSNET_NOALLOC_SCRATCH_BYTES)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED,
                "problem needs " + std::to_string(need) + " bytes of scratch; the fixed "
                "scratch array of rosnet_tensordot_noalloc holds " +
                std::to_string((size_t)ROSNET_NOALLOC_SCRATCH_BYTES) + " bytes");
    C->stream = s;
    return ROSNET_OK;
    RN_API_END
}
