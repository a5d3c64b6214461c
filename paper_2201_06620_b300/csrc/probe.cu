// Peak-rate probes: microkernels that measure the rate this GPU sustains for
// each kind of arithmetic the contraction kernels use, so that their
// roofline fractions can be stated against measured numbers instead of unit
// counts times clocks.
//
//   ROSNET_PROBE_FFMA   FP32 fused multiply-adds on the CUDA cores (the
//                       packed and tiled complex64 kernels)
//   ROSNET_PROBE_DFMA   FP64 fused multiply-adds (the complex128 kernels)
//   ROSNET_PROBE_TF32   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, FP32
//                       accumulators in tensor memory (TF32 and 3xTF32 modes)
//   ROSNET_PROBE_BF16   tcgen05.mma kind::f16 with bf16 operands, M = 128,
//                       N = 256, K = 16 (3xBF16 mode)
//
// The FMA probes run 16 independent chains per thread at full occupancy; the
// MMA probes issue back-to-back MMAs from one thread per SM on operands
// resident in shared memory, so only the tensor pipe limits them.  Each
// probe is launched once to warm up and once timed with CUDA events.
#include <cuda_runtime.h>

#include <cstring>

#include "gett_common.cuh"

namespace rosnet {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T a, T b, int iters, T *sink) {
    T x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += x[j];
    if (s == (T)-12345.0) *sink = s;   // never true; keeps every chain live
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major shared-memory operand descriptor, 64-byte swizzle, 8-row groups
// 512 bytes apart (the layout of the tensor-core GEMM's stages).
__device__ __forceinline__ uint64_t probe_sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

constexpr int kProbeM = 128, kProbeN = 256;
constexpr size_t kProbeSmem = 128 * 1024;   // more than half of an SM's: one CTA per SM

// BF16 = false: kind::tf32 (K = 8 per MMA); true: kind::f16 with bf16 (K = 16).
template <bool BF16>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int iters, long long budget, int32_t *status) {
    extern __shared__ unsigned char raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    // operands: A 128 rows x 64 bytes, B 256 rows x 64 bytes (values do not
    // matter for the rate; zeros)
    constexpr int kBytes = (kProbeM + kProbeN) * 64;
    for (int i = threadIdx.x; i < kBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t sa = su32(sm), sb = sa + kProbeM * 64;
        const uint32_t id = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                            ((uint32_t)(kProbeN >> 3) << 17) | ((uint32_t)(kProbeM >> 4) << 24);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {   // two 32-byte K slices of the 64-byte rows
                const uint64_t ad = probe_sdesc(sa + ks * 32), bd = probe_sdesc(sb + ks * 32);
                const uint32_t acc = (i | ks) ? 1u : 0u;
                if (BF16)
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(id), "r"(acc)
                        : "memory");
                else
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(id), "r"(acc)
                        : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar))
                     : "memory");
        // bounded wait for every MMA of this thread
        const long long t0 = clock64();
        uint32_t done = 0;
        while (!done) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                " selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(su32(&bar))
                : "memory");
            if (!done && clock64() - t0 > budget) {
                atomicExch(status, kDevErrTimeout);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

}  // namespace
}  // namespace rosnet

using namespace rosnet;

extern "C" rosnet_status rosnet_probe_peak(int32_t kind, void *stream, double *flops, double *ms) {
    RN_API_BEGIN
    if (!flops || !ms) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = num_sms();
    DevBuf sink(16, s);   // [0, 8): the FMA probes' sink; [8, 12): the MMA probes' status
    int32_t *status = (int32_t *)((char *)sink.p + 8);
    RN_CHECK_CUDA(cudaMemsetAsync(sink.p, 0, 16, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RN_CHECK_CUDA(cudaEventCreate(&e0));
    RN_CHECK_CUDA(cudaEventCreate(&e1));
    double fl = 0;
    auto run = [&](bool timed) {
        if (timed) RN_CHECK_CUDA(cudaEventRecord(e0, s));
        switch (kind) {
            case ROSNET_PROBE_FFMA: {
                const int blocks = sms * 8, iters = 1 << 16;
                fma_probe_kernel<float><<<blocks, 256, 0, s>>>(0.999f, 1e-3f, iters, (float *)sink.p);
                fl = 2.0 * 16 * (double)iters * blocks * 256;
                break;
            }
            case ROSNET_PROBE_DFMA: {
                const int blocks = sms * 8, iters = 1 << 11;
                fma_probe_kernel<double><<<blocks, 256, 0, s>>>(0.999, 1e-3, iters, (double *)sink.p);
                fl = 2.0 * 16 * (double)iters * blocks * 256;
                break;
            }
            case ROSNET_PROBE_TF32:
            case ROSNET_PROBE_BF16: {
                const bool bf = kind == ROSNET_PROBE_BF16;
                const int iters = 1 << 15;
                auto kern = bf ? mma_probe_kernel<true> : mma_probe_kernel<false>;
                RN_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kProbeSmem));
                kern<<<sms, 128, kProbeSmem, s>>>(iters, 4000000000LL, status);
                fl = 2.0 * kProbeM * kProbeN * (bf ? 16 : 8) * 2.0 * (double)iters * sms;
                break;
            }
            default: RN_FAIL(ROSNET_ERR_INVALID_ARG, "unknown probe kind");
        }
        g_launches++;
        RN_CHECK_CUDA(cudaGetLastError());
        if (timed) RN_CHECK_CUDA(cudaEventRecord(e1, s));
    };
    try {
        run(false);
        run(true);
        RN_CHECK_CUDA(cudaEventSynchronize(e1));
        float t = 0;
        RN_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
        *ms = t;
        *flops = fl;
        int32_t st = 0;
        RN_CHECK_CUDA(cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost));
        if (st != 0) RN_FAIL(ROSNET_ERR_TIMEOUT, "a probe's bounded wait gave up");
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ROSNET_OK;
    RN_API_END
}
