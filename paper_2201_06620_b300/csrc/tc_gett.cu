// The blocked pairwise tensordot on the 5th-generation tensor cores.
//
// Complex64 block products run as real tcgen05 GEMMs with FP32 accumulators
// in tensor memory (TMEM) that persist across the whole contracted-index loop,
// i.e. across every matched block pair of the output tile (Sec. II-C steps
// 3-4: all partial products of an output block are summed in place, in any
// order, Sec. IV-A).  With planar operands the complex product is four real
// products:
//     Cr += Ar*Br + (-Ai)*Bi        (the minus is the MMA's negate-A bit)
//     Ci += Ar*Bi + Ai*Br
// Precision modes (each operand element x is converted while it is staged):
//   TF32    x -> tf32(x)                                  1 product per term
//   TF32X3  x = big + small, both tf32;  big*big + big*small + small*big
//   BF16X3  x = hi + lo, both bf16;      hi*hi + hi*lo + lo*hi  (kind::f16)
//
// CTA = 256 threads: warps 0-3 gather the A and B tiles of each k-stage
// through the offset tables into the 64-byte-swizzled K-major layout the MMA
// reads (any axis permutation and blocking); one thread of warp 4 issues the
// MMAs; warps 4-7 move the accumulators TMEM -> registers -> C.  Stages are
// handed over with mbarriers.  Every wait is bounded: on timeout the kernel
// records kDevErrTimeout in a device status word, stops, waits for its own
// MMAs, frees its TMEM and returns (rosnet_sync reports ROSNET_ERR_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gett_common.cuh"

namespace rosnet {

__device__ int32_t g_dev_status = 0;

namespace tc {

constexpr int BM = 128, BN = 128;
constexpr int ROWB = 64;                  // bytes of one K-row of a stage (64B swizzle)
constexpr int NTHREADS = 256;
constexpr int NPROD = 128;                // producer threads (warps 0-3)
constexpr long long kWaitBudget = 4000000000LL;   // cycles (~2 s at 2 GHz)

enum Mode : int { kTF32 = 0, kTF32x3 = 1, kBF16x3 = 2 };

template <int MODE>
struct Cfg {
    static constexpr int ESZ = MODE == kBF16x3 ? 2 : 4;       // bytes per staged element
    static constexpr int BK = ROWB / ESZ;                     // k per stage (16 or 32)
    static constexpr int NARR = MODE == kTF32 ? 2 : 4;        // arrays per operand
    static constexpr int ARR_A = BM * ROWB, ARR_B = BN * ROWB;  // bytes of one array
    static constexpr int STAGE = NARR * (ARR_A + ARR_B);
    static constexpr int STAGES = MODE == kTF32 ? 6 : 3;
    static constexpr int KSTEP = 32 / ESZ;                    // k of one MMA (8 tf32 / 16 bf16)
    static constexpr int KSTEPS = BK / KSTEP;                 // MMAs per product per stage (2)
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024;  // + alignment slack
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity`; false on timeout, or on abort by
// another thread when `honor_abort` is set.
__device__ __noinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort,
                                       bool honor_abort = true) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity)) {
        if (honor_abort && *abort) return false;
        if (clock64() - t0 > kWaitBudget) {
            atomicExch(&g_dev_status, kDevErrTimeout);
            *abort = 1;
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)4 << 61;                     // swizzle: 64B
    return d;
}

// Instruction descriptor: FP32 accumulator, M=128, N=128, both K-major.
template <int MODE>
__host__ __device__ constexpr uint32_t idesc(bool negate_a) {
    return (1u << 4)                                          // D: f32
           | ((MODE == kBF16x3 ? 1u : 2u) << 7)               // A: bf16 (kind::f16) / tf32
           | ((MODE == kBF16x3 ? 1u : 2u) << 10)              // B
           | ((negate_a ? 1u : 0u) << 13)                     // negate A
           | ((uint32_t)(BN >> 3) << 17)                      // N
           | ((uint32_t)(BM >> 4) << 24);                     // M
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    if (MODE == kBF16x3)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Byte offset of element (row r, k) of one array (64-byte rows, 64B swizzle).
__device__ __forceinline__ uint32_t swz(int r, int kbyte) {
    const int c = kbyte >> 4;
    return (uint32_t)(r * ROWB + ((c ^ ((r >> 1) & 3)) << 4) + (kbyte & 15));
}

// Stage one element x of an operand row into its arrays (re planes: arrays
// 0[,1]; im planes: arrays 1 or 2[,3]).
template <int MODE>
__device__ __forceinline__ void put(unsigned char *arr0, int arr_bytes, int plane, int r, int k, float x) {
    constexpr int ESZ = Cfg<MODE>::ESZ;
    const uint32_t off = swz(r, k * ESZ);
    if (MODE == kTF32) {
        *reinterpret_cast<uint32_t *>(arr0 + plane * arr_bytes + off) = to_tf32(x);
    } else if (MODE == kTF32x3) {
        const uint32_t big = to_tf32(x);
        const uint32_t small = to_tf32(x - __uint_as_float(big));
        *reinterpret_cast<uint32_t *>(arr0 + (2 * plane) * arr_bytes + off) = big;
        *reinterpret_cast<uint32_t *>(arr0 + (2 * plane + 1) * arr_bytes + off) = small;
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(arr0 + (2 * plane) * arr_bytes + off) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(arr0 + (2 * plane + 1) * arr_bytes + off) = lo;
    }
}

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gett_kernel(const __grid_constant__ GroupArgs g) {
    using C_ = Cfg<MODE>;
    constexpr int BK = C_::BK, STAGES = C_::STAGES, NARR = C_::NARR;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *dsm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ GettDesc sd;
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int64_t s_arow[BM], s_brow[BN];   // element offsets of the tile's rows (-1: outside)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        load_desc(g, sd);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], NPROD);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {   // the MMA warp owns the accumulators: 2 x 128 columns (Cr, Ci)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                         su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();   // descriptor visible
    const int64_t tile = (int64_t)blockIdx.x - sd.tile_begin;
    const int64_t m0 = (tile % sd.tiles_m) * BM, n0 = (tile / sd.tiles_m) * BN;
    const int64_t M = sd.M, N = sd.N, K = sd.K;
    const int nkt = (int)((K + BK - 1) / BK);
    if (tid < BM) s_arow[tid] = (m0 + tid < M) ? sd.offAM[m0 + tid] : -1;
    else if (tid < BM + BN) s_brow[tid - BM] = (n0 + tid - BM < N) ? sd.offBN[n0 + tid - BM] : -1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp < 4) {
        // ------------------------------------------------------------ producers
        const bool amf = sd.flags & kFlagAMFast, bnf = sd.flags & kFlagBNFast;
        const float *__restrict__ A = (const float *)sd.a;
        const float *__restrict__ B = (const float *)sd.b;
        const int64_t ap = sd.a_plane, bp = sd.b_plane;
        const int pt = tid;   // 0..127
        // a "fast" operand is read one row per thread over all k of the stage;
        // otherwise one k per thread over BK rows spaced NPROD/BK apart
        constexpr int RSTEP = NPROD / BK;
        for (int kt = 0; kt < nkt; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait(&empty_bar[s], ((kt / STAGES) & 1) ^ 1, &abort_flag)) break;
            unsigned char *sa = dsm + (size_t)s * C_::STAGE;
            unsigned char *sb = sa + NARR * C_::ARR_A;
            const int64_t k0 = (int64_t)kt * BK;
            // A tile
            if (amf) {
                const int r = pt;
                const int64_t ro = s_arow[r];
#pragma unroll 4
                for (int kk = 0; kk < BK; ++kk) {
                    const int64_t k = k0 + kk;
                    float xr = 0.f, xi = 0.f;
                    if (ro >= 0 && k < K) {
                        const int64_t o = ro + __ldg(sd.offAK + k);
                        xr = __ldg(A + o);
                        xi = __ldg(A + o + ap);
                    }
                    put<MODE>(sa, C_::ARR_A, 0, r, kk, xr);
                    put<MODE>(sa, C_::ARR_A, 1, r, kk, xi);
                }
            } else {
                const int kk = pt % BK;
                const int64_t k = k0 + kk;
                const int64_t ko = k < K ? __ldg(sd.offAK + k) : 0;
#pragma unroll 4
                for (int j = 0; j < BK; ++j) {
                    const int r = pt / BK + j * RSTEP;
                    const int64_t ro = s_arow[r];
                    float xr = 0.f, xi = 0.f;
                    if (ro >= 0 && k < K) {
                        const int64_t o = ro + ko;
                        xr = __ldg(A + o);
                        xi = __ldg(A + o + ap);
                    }
                    put<MODE>(sa, C_::ARR_A, 0, r, kk, xr);
                    put<MODE>(sa, C_::ARR_A, 1, r, kk, xi);
                }
            }
            // B tile
            if (bnf) {
                const int r = pt;
                const int64_t ro = s_brow[r];
#pragma unroll 4
                for (int kk = 0; kk < BK; ++kk) {
                    const int64_t k = k0 + kk;
                    float xr = 0.f, xi = 0.f;
                    if (ro >= 0 && k < K) {
                        const int64_t o = ro + __ldg(sd.offBK + k);
                        xr = __ldg(B + o);
                        xi = __ldg(B + o + bp);
                    }
                    put<MODE>(sb, C_::ARR_B, 0, r, kk, xr);
                    put<MODE>(sb, C_::ARR_B, 1, r, kk, xi);
                }
            } else {
                const int kk = pt % BK;
                const int64_t k = k0 + kk;
                const int64_t ko = k < K ? __ldg(sd.offBK + k) : 0;
#pragma unroll 4
                for (int j = 0; j < BK; ++j) {
                    const int r = pt / BK + j * RSTEP;
                    const int64_t ro = s_brow[r];
                    float xr = 0.f, xi = 0.f;
                    if (ro >= 0 && k < K) {
                        const int64_t o = ro + ko;
                        xr = __ldg(B + o);
                        xi = __ldg(B + o + bp);
                    }
                    put<MODE>(sb, C_::ARR_B, 0, r, kk, xr);
                    put<MODE>(sb, C_::ARR_B, 1, r, kk, xi);
                }
            }
            fence_proxy_async();   // generic-proxy stores -> visible to the MMA (async proxy)
            mbar_arrive(&full_bar[s]);
        }
    } else if (warp == 4) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t dr = tmem, di = tmem + BN;   // Cr: columns [0,128), Ci: [128,256)
            for (int kt = 0; kt < nkt; ++kt) {
                const int s = kt % STAGES;
                if (!mbar_wait(&full_bar[s], (kt / STAGES) & 1, &abort_flag)) break;
                tc_fence_after();
                const uint32_t sa = su32(dsm + (size_t)s * C_::STAGE);
                const uint32_t sb = sa + NARR * C_::ARR_A;
#pragma unroll
                for (int ks = 0; ks < C_::KSTEPS; ++ks) {
                    const uint32_t kb = ks * 32;   // byte offset of this MMA's K slice
                    auto A_ = [&](int arr) { return sdesc(sa + arr * C_::ARR_A + kb); };
                    auto B_ = [&](int arr) { return sdesc(sb + arr * C_::ARR_B + kb); };
                    const uint32_t first = (kt == 0 && ks == 0) ? 0u : 1u;
                    if (MODE == kTF32) {
                        // arrays: 0 = re, 1 = im
                        mma<MODE>(dr, A_(0), B_(0), idesc<MODE>(false), first);
                        mma<MODE>(dr, A_(1), B_(1), idesc<MODE>(true), 1u);
                        mma<MODE>(di, A_(0), B_(1), idesc<MODE>(false), first);
                        mma<MODE>(di, A_(1), B_(0), idesc<MODE>(false), 1u);
                    } else {
                        // arrays: 0 = re big/hi, 1 = re small/lo, 2 = im big/hi, 3 = im small/lo
                        // small terms first, then the big*big term
                        mma<MODE>(dr, A_(0), B_(1), idesc<MODE>(false), first);
                        mma<MODE>(dr, A_(1), B_(0), idesc<MODE>(false), 1u);
                        mma<MODE>(dr, A_(2), B_(3), idesc<MODE>(true), 1u);
                        mma<MODE>(dr, A_(3), B_(2), idesc<MODE>(true), 1u);
                        mma<MODE>(dr, A_(0), B_(0), idesc<MODE>(false), 1u);
                        mma<MODE>(dr, A_(2), B_(2), idesc<MODE>(true), 1u);
                        mma<MODE>(di, A_(0), B_(3), idesc<MODE>(false), first);
                        mma<MODE>(di, A_(1), B_(2), idesc<MODE>(false), 1u);
                        mma<MODE>(di, A_(2), B_(1), idesc<MODE>(false), 1u);
                        mma<MODE>(di, A_(3), B_(0), idesc<MODE>(false), 1u);
                        mma<MODE>(di, A_(0), B_(2), idesc<MODE>(false), 1u);
                        mma<MODE>(di, A_(2), B_(0), idesc<MODE>(false), 1u);
                    }
                }
                mma_commit(&empty_bar[s]);   // frees the stage when these MMAs are done
            }
            mma_commit(&done_bar);           // all MMAs issued by this thread are complete
        }
        __syncwarp();
    }

    if (warp >= 4) {
        // ------------------------------------------------------------ epilogue
        // wait for every MMA even after an abort: TMEM must not be freed under them
        bool ok = mbar_wait(&done_bar, 0, &abort_flag, false);
        ok = __all_sync(0xffffffffu, ok) && !abort_flag;
        tc_fence_after();
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int r = q * 32 + lane;            // output row of this thread
        const bool rok = ok && (m0 + r < M) && nkt > 0;
        const int64_t cm = (m0 + r < M) ? sd.offCM[m0 + r] : 0;   // C offset of row r
        float *__restrict__ C = (float *)sd.c;
        const int64_t cp = sd.c_plane;
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float vr[16], vi[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c0, vr);
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + BN + c0, vi);
                if (rok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t n = n0 + c0 + j;
                        if (n < N) {
                            const int64_t o = cm + __ldg(sd.offCN + n);
                            C[o] = vr[j];
                            C[o + cp] = vi[j];
                        }
                    }
                }
            }
        }
        // no contracted index at all: the result is zero
        if (ok && nkt == 0 && m0 + r < M)
            for (int64_t n = n0; n < n0 + BN && n < N; ++n) {
                const int64_t o = cm + sd.offCN[n];
                C[o] = 0.f;
                C[o + cp] = 0.f;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool tc_mode_of(int precision, int *mode) {
    switch (precision) {
        case ROSNET_PREC_TF32: *mode = tc::kTF32; return true;
        case ROSNET_PREC_TF32X3: *mode = tc::kTF32x3; return true;
        case ROSNET_PREC_BF16X3: *mode = tc::kBF16x3; return true;
        default: return false;
    }
}

template <int MODE>
static void launch_tc_mode(dim3 grid, const GroupArgs &ga, cudaStream_t s) {
    using C_ = tc::Cfg<MODE>;
    static bool attr_set = false;
    if (!attr_set) {
        RN_CHECK_CUDA(cudaFuncSetAttribute(tc::tc_gett_kernel<MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_::SMEM));
        attr_set = true;
    }
    tc::tc_gett_kernel<MODE><<<grid, tc::NTHREADS, C_::SMEM, s>>>(ga);
}

void launch_tc_group(int mode, const GroupArgs &ga, int64_t ctas, cudaStream_t s) {
    if (ctas <= 0) return;
    if (ctas > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "too many tiles in one launch");
    dim3 grid((unsigned)ctas);
    switch (mode) {
        case tc::kTF32: launch_tc_mode<tc::kTF32>(grid, ga, s); break;
        case tc::kTF32x3: launch_tc_mode<tc::kTF32x3>(grid, ga, s); break;
        default: launch_tc_mode<tc::kBF16x3>(grid, ga, s); break;
    }
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

int tc_tile_m() { return tc::BM; }
int tc_tile_n() { return tc::BN; }

// Read and clear the device status word (0 = no kernel gave up a wait).
int32_t take_device_status() {
    int32_t v = 0, z = 0;
    RN_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(v)));
    if (v) RN_CHECK_CUDA(cudaMemcpyToSymbol(g_dev_status, &z, sizeof(z)));
    return v;
}

}  // namespace rosnet
