// rosnet_tensordot_noalloc: the pairwise tensordot for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they contract: code that runs inside a framework that owns all device
// memory and forbids foreign allocations, real-time or embedded callers with
// a fixed, pre-committed memory budget, and callers on a path where an
// allocation could block or fail unpredictably.  They pass inputs and an
// already created output tensor; the scratch the kernels need (offset tables
// and split-K partial sums) lives in one file-scope device array of fixed
// size instead of coming from an allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace rosnet {

void check_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axes_a,
                     const int *axes_b, int *axa, int *axb, int &rc, int64_t *shc, int64_t *blc);
int check_precision(const rosnet_opts *opts, int dtype);
size_t tensordot_into_ws(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axa,
                         const int *axb, rosnet_btensor C, int precision, void *ws,
                         size_t ws_bytes, cudaStream_t s);

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ROSNET_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
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
    if (C == A || C == B || C->data == A->data || C->data == B->data)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "the output may not alias an operand");
    if (C->dtype != A->dtype) RN_FAIL(ROSNET_ERR_DTYPE, "output dtype differs from the operands'");
    if (C->lay.rank != rc) RN_FAIL(ROSNET_ERR_SHAPE, "output rank does not match the result");
    for (int i = 0; i < rc; ++i) {
        if (C->lay.shape[i] != shc[i]) RN_FAIL(ROSNET_ERR_SHAPE, "output shape does not match the result");
        if (C->lay.block[i] != blc[i])
            RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "output block shape does not match the result");
    }
    const int prec = check_precision(opts, A->dtype);
    void *ws = scratch_on_current_device();
    const size_t need = tensordot_into_ws(A, B, naxes, axa, axb, C, prec, ws,
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
