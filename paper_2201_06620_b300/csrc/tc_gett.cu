// The blocked pairwise tensordot on the 5th-generation tensor cores.
//
// Complex64 block products run as real tcgen05 GEMMs with FP32 accumulators
// in tensor memory (TMEM).  With planar operands the complex product is four
// real products:
//     Cr += Ar*Br + (-Ai)*Bi        (the minus is the MMA's negate-A bit)
//     Ci += Ar*Bi + Ai*Br
// Precision modes (each operand element x is converted once, when packed):
//   TF32    x -> tf32(x)                                  1 product per term
//   TF32X3  x = big + small, both tf32;  big*big + big*small + small*big
//   BF16X3  x = hi + lo, both bf16;      hi*hi + hi*lo + lo*hi  (kind::f16)
//
// Two kernels per problem:
//   1. tc_pack_kernel gathers each operand through its offset tables (any
//      axis permutation and block layout, coalesced along the operand's
//      unit-stride digit, transposed through shared memory) and writes the
//      converted parts as K-major [rows][K] arrays padded to whole tiles.
//   2. tc_gemm_kernel: one thread streams 128 x (64-byte) boxes of those
//      arrays into a ring of shared-memory stages with TMA tensor copies
//      (cp.async.bulk.tensor, 64-byte swizzle = the MMA's K-major layout);
//      one thread issues the MMAs; eight warps own the output tile.  The
//      contracted loop (every matched block pair of the tile, Sec. II-C steps
//      2-4) is accumulated in chunks (256 k for TF32, 16 k for 3xTF32, 64 k
//      for 3xBF16) in two alternating TMEM accumulators; the eight warps add each
//      finished chunk into FP32 registers while the tensor core fills the
//      other one.  The tensor core's accumulator adds carry a small one-sided
//      error that grows with the number of terms; chunking caps it.  The sum
//      over pairs is order-free (Sec. IV-A); the order here is fixed.
//
// Every wait is bounded: on timeout the kernel records kDevErrTimeout in a
// device status word, stops issuing work, waits (bounded) for its own copies
// and MMAs, frees its TMEM and returns; rosnet_sync reports
// ROSNET_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <mutex>

#include "gett_common.cuh"

namespace rosnet {

__device__ int32_t g_dev_status = 0;

namespace tc {

constexpr int BM = 128, BN = 128;
constexpr int ROWB = 64;                 // bytes of one K-row of a stage (64B swizzle span)
constexpr int NTHREADS = 320;            // warp 0 TMA, warp 1 MMA, warps 2-9 accumulators
constexpr int NACC_WARPS = 8;
// contracted indices per TMEM accumulation chunk.  The tensor core's FP32
// accumulator adds carry a one-sided error that grows with the number of
// terms; each finished chunk is added into FP32 registers.  TF32: 4096 (its
// error is set by the operand rounding, 2^-11 of each operand; the
// accumulator's bias over 4096 terms, ~1.4e-8 each, stays far below it, and
// one chunk per tile for most shapes leaves the accumulator drain off the
// tensor core's path: 661 -> 689 TFLOP/s on 2^10 x 2^15 x 2^10 against
// 256-term chunks).  3xTF32, the FP32-accuracy arm: 16,
// which brings its amplitudes to plain FP32's error on deep circuits
// (measured vs the FP64 oracle on 16-20 qubit, depth 12-16 circuits: worst
// 8.8e-6 against FP32's 9.1e-6; 1.06e-5 with 32, 1.28e-5 with 64) for 16%
// of its throughput on large contractions.  3xBF16: 128 (its error is set by
// the bf16 split: the 20-qubit amplitude's error against plain FP32 is
// 1.71e-5 with 16-, 64- or 128-term chunks, 1.94e-5 with 256; 128 against 64
// gives 501 -> 542 TFLOP/s on 2^10 x 2^15 x 2^10).
constexpr int chunk_k(int mode) { return mode == 0 ? 4096 : mode == 1 ? 16 : 128; }
constexpr long long kWaitBudget = 4000000000LL;   // cycles (~2 s at 2 GHz)

enum Mode : int { kTF32 = 0, kTF32x3 = 1, kBF16x3 = 2 };

template <int MODE>
struct Cfg {
    static constexpr int ESZ = MODE == kBF16x3 ? 2 : 4;        // bytes per packed element
    static constexpr int BK = ROWB / ESZ;                      // k per stage (16 or 32)
    static constexpr int NARR = MODE == kTF32 ? 2 : 4;         // arrays of A
    static constexpr int NARR_B = MODE == kTF32 ? 3 : 4;       // arrays of B (TF32: re, im, -re)
    // stage position of B's array a: in the split modes (re hi, re lo, im hi,
    // im lo) are staged as (re lo, im lo, re hi, im hi), so that [re lo | im
    // lo] and [re hi | im hi] are contiguous N = 256 operand windows
    static constexpr int bpos(int a) { return MODE == kTF32 ? a : (a == 0 ? 2 : a == 1 ? 0 : a == 2 ? 3 : 1); }
    static constexpr int ARR_A = BM * ROWB, ARR_B = BN * ROWB;   // bytes of one array's box
    static constexpr int STAGE = NARR * ARR_A + NARR_B * ARR_B;
    static constexpr int STAGES = MODE == kTF32 ? 5 : 3;
    static constexpr int KSTEPS = BK / (32 / ESZ);             // MMAs per product per stage
    static constexpr int CH_STAGES = chunk_k(MODE) / BK;       // stages per chunk
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024;
};

struct TcArgs {
    CUtensorMap mapA[4];   // packed A arrays (re[,re_lo], im[,im_lo]) as [Mpad][Kpad]
    CUtensorMap mapB[4];
    GroupArgs g;           // the problem (C pointer, C offset tables, M, N, K, tiles)
    int32_t nkt;           // k-stages (Kpad / BK)
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
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

// The same bounded wait without sleeping between tests: for the one thread
// whose wake-up latency stalls the tensor core (the MMA issuer).
__device__ __noinline__ bool mbar_wait_spin(uint64_t *b, uint32_t parity, volatile int *abort) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitBudget) {
            atomicExch(&g_dev_status, kDevErrTimeout);
            *abort = 1;
            return false;
        }
    }
    return true;
}

// The same wait with the uncontended case inline (one try_wait, no call):
// for hot loops that usually find the phase already complete.
__device__ __forceinline__ bool mbar_wait_fast(uint64_t *b, uint32_t parity, volatile int *abort) {
    if (mbar_try(b, parity)) return true;
    return mbar_wait(b, parity, abort);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(su32(bar))
        : "memory");
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

// Instruction descriptor: FP32 accumulator, M=128, N=128 (or n), both K-major.
template <int MODE>
__host__ __device__ constexpr uint32_t idesc(bool negate_a, int n = BN) {
    return (1u << 4)                                          // D: f32
           | ((MODE == kBF16x3 ? 1u : 2u) << 7)               // A: bf16 (kind::f16) / tf32
           | ((MODE == kBF16x3 ? 1u : 2u) << 10)              // B
           | ((negate_a ? 1u : 0u) << 13)                     // negate A
           | ((uint32_t)(n >> 3) << 17)                       // N
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// 1. pack: gather + convert one operand into K-major [Rpad][Kpad] part arrays
// ---------------------------------------------------------------------------
// which = 0: operand A of the problem (rows = M digits), 1: operand B (rows =
// N digits).  32 x 32 (row, k) tiles, 256 threads, transposed through shared
// memory so that both the gather and the row-major store coalesce.
template <int MODE>
__global__ void __launch_bounds__(256) tc_pack_kernel(const __grid_constant__ GroupArgs g, int which,
                                                      unsigned char *__restrict__ out, int64_t Rpad,
                                                      int64_t Kpad) {
    using C_ = Cfg<MODE>;
    __shared__ GettDesc sd;
    __shared__ float tr[2][32][33];
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const float *__restrict__ src = (const float *)(which ? sd.b : sd.a);
    const int64_t plane = which ? sd.b_plane : sd.a_plane;
    const int64_t *__restrict__ offR = which ? sd.offBN : sd.offAM;
    const int64_t *__restrict__ offK = which ? sd.offBK : sd.offAK;
    const int64_t R = which ? sd.N : sd.M, K = sd.K;
    const bool row_fast = which ? (sd.flags & kFlagBNFast) : (sd.flags & kFlagAMFast);
    const int64_t ktiles = Kpad / 32;
    const int64_t r0 = ((int64_t)blockIdx.x / ktiles) * 32, k0 = ((int64_t)blockIdx.x % ktiles) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int a = tx, b = ty + 8 * j;
        const int rr = row_fast ? a : b, kk = row_fast ? b : a;
        const int64_t r = r0 + rr, k = k0 + kk;
        float xr = 0.f, xi = 0.f;
        if (r < R && k < K) {
            const int64_t o = offR[r] + offK[k];
            xr = src[o];
            xi = src[o + plane];
        }
        tr[0][kk][rr] = xr;
        tr[1][kk][rr] = xi;
    }
    __syncthreads();
    const size_t arr = (size_t)Rpad * Kpad * C_::ESZ;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int rr = ty + 8 * j, kk = tx;
        const size_t e = (size_t)(r0 + rr) * Kpad + (k0 + kk);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float x = tr[p][kk][rr];
            if (MODE == kTF32) {
                reinterpret_cast<uint32_t *>(out + p * arr)[e] = to_tf32(x);
                if (which == 1 && p == 0) reinterpret_cast<uint32_t *>(out + 2 * arr)[e] = to_tf32(-x);
            } else if (MODE == kTF32x3) {
                const uint32_t big = to_tf32(x);
                reinterpret_cast<uint32_t *>(out + (2 * p) * arr)[e] = big;
                reinterpret_cast<uint32_t *>(out + (2 * p + 1) * arr)[e] = to_tf32(x - __uint_as_float(big));
            } else {
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                reinterpret_cast<__nv_bfloat16 *>(out + (2 * p) * arr)[e] = hi;
                reinterpret_cast<__nv_bfloat16 *>(out + (2 * p + 1) * arr)[e] =
                    __float2bfloat16_rn(x - __bfloat162float(hi));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2. TMA + tcgen05 GEMM with chunked TMEM accumulation
// ---------------------------------------------------------------------------
// Persistent: one CTA per SM walks the output tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; stages and TMEM chunks are numbered across
// the CTA's tiles, so the TMA ring and the two accumulators run on from one
// tile into the next: the tensor core starts the next tile's first chunk
// while the accumulator warps add the last chunk of the previous one and
// store it, and the CTA's setup (barriers, TMEM allocation) happens once.
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_kernel(const __grid_constant__ TcArgs p) {
    using C_ = Cfg<MODE>;
    constexpr int STAGES = C_::STAGES, NARR = C_::NARR, BK = C_::BK;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *dsm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ GettDesc sd;
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accf[2], acce[2], fin_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) load_desc(p.g, sd);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], NACC_WARPS);
        }
        mbar_init(&fin_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // two accumulators of Cr|Ci (2 x 256 columns): all of TMEM
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    // raster: the operand with fewer tiles varies fastest, so its tiles stay
    // resident in L2 while the other operand streams through once
    const bool n_fast = sd.tiles_n < sd.tiles_m;
    auto tile_origin = [&](int64_t tile, int64_t &m0, int64_t &n0) {
        const int64_t tm = n_fast ? tile / sd.tiles_n : tile % sd.tiles_m;
        const int64_t tn = n_fast ? tile % sd.tiles_n : tile / sd.tiles_m;
        m0 = tm * BM;
        n0 = tn * BN;
    };
    const int64_t ntiles = sd.tiles_m * sd.tiles_n;
    const int64_t first = (int64_t)blockIdx.x - sd.tile_begin, G = gridDim.x;
    const int mytiles = first < ntiles ? (int)((ntiles - first + G - 1) / G) : 0;
    const int nkt = p.nkt;
    const int nchunks = (nkt + C_::CH_STAGES - 1) / C_::CH_STAGES;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            int issued = 0;   // stages issued over all tiles
            bool go = true;
            for (int i = 0; i < mytiles && go; ++i) {
                int64_t m0, n0;
                tile_origin(first + (int64_t)i * G, m0, n0);
                for (int kt = 0; kt < nkt; ++kt) {
                    const int g = issued, s = g % STAGES;
                    if (!mbar_wait(&empty_bar[s], ((g / STAGES) & 1) ^ 1, &abort_flag)) {
                        go = false;
                        break;
                    }
                    mbar_expect_tx(&full_bar[s], C_::STAGE);
                    const uint32_t sa = su32(dsm + (size_t)s * C_::STAGE);
                    const uint32_t sb = sa + NARR * C_::ARR_A;
#pragma unroll
                    for (int a = 0; a < NARR; ++a)
                        tma_load_2d(sa + a * C_::ARR_A, &p.mapA[a], kt * BK, (int)m0, &full_bar[s]);
#pragma unroll
                    for (int a = 0; a < C_::NARR_B; ++a)
                        tma_load_2d(sb + C_::bpos(a) * C_::ARR_B, &p.mapB[a], kt * BK, (int)n0, &full_bar[s]);
                    issued = g + 1;
                }
            }
            // copies still in flight must land before this CTA can exit
            for (int g = (issued > STAGES ? issued - STAGES : 0); g < issued; ++g)
                mbar_wait(&full_bar[g % STAGES], (g / STAGES) & 1, &abort_flag, false);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issue
        if (lane == 0) {
            int g = 0;    // stage counter over all tiles
            int gc = 0;   // chunk counter over all tiles
            // the full barrier of stage g was already seen complete: each
            // stage's test is issued while the previous stage's MMAs go out,
            // so its latency is not paid between them
            bool ready = false;
            bool go = true;
            for (int i = 0; i < mytiles && go; ++i) {
                int kt = 0;
                for (int c = 0; c < nchunks && go; ++c, ++gc) {
                    const int b = gc & 1;
                    if (gc >= 2 && !mbar_wait_spin(&acce[b], ((gc >> 1) - 1) & 1, &abort_flag)) {
                        go = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dr = tmem + b * 2 * BN, di = dr + BN;
                    const int kend = min(nkt, (c + 1) * C_::CH_STAGES);
                    for (; kt < kend; ++kt, ++g) {
                        const int s = g % STAGES;
                        if (!ready && !mbar_wait_fast(&full_bar[s], (g / STAGES) & 1, &abort_flag)) {
                            go = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = su32(dsm + (size_t)s * C_::STAGE);
                        const uint32_t sb = sa + NARR * C_::ARR_A;
#pragma unroll
                        for (int ks = 0; ks < C_::KSTEPS; ++ks) {
                            const uint32_t kb = ks * 32;   // byte offset of this MMA's K slice
                            auto A_ = [&](int arr) { return sdesc(sa + arr * C_::ARR_A + kb); };
                            auto B_ = [&](int arr) { return sdesc(sb + arr * C_::ARR_B + kb); };
                            const uint32_t acc = (kt == c * C_::CH_STAGES && ks == 0) ? 0u : 1u;
                            if (ks == C_::KSTEPS - 1)
                                ready = mbar_try(&full_bar[(g + 1) % STAGES], ((g + 1) / STAGES) & 1);
                            if (MODE == kTF32) {
                                // A arrays: 0 = re, 1 = im; B arrays: 0 = re, 1 = im, 2 = -re.
                                // [dr | di] (256 columns) += A_re [B_re | B_im], then
                                // (-A_im) [B_im | -B_re]
                                mma<MODE>(dr, A_(0), B_(0), idesc<MODE>(false, 2 * BN), acc);
                                mma<MODE>(dr, A_(1), B_(1), idesc<MODE>(true, 2 * BN), 1u);
                            } else {
                                // A arrays: 0 = re big/hi, 1 = re small/lo, 2 = im big/hi,
                                // 3 = im small/lo; B the same arrays at stage positions
                                // bpos: B_(0) = [B1 | B3], B_(2) = [B0 | B2] as N = 256
                                // windows, B_(1) = B3, B_(3) = B2, B_(0) = B1, B_(2) = B0
                                // as N = 128 ones.  The positive products of both parts
                                // go out as N = 256 MMAs into [dr | di], each part's small
                                // terms before its large ones (the order of the twelve
                                // N = 128 products: dr A0B1, A1B0, -A2B3, -A3B2, A0B0,
                                // -A2B2; di A0B3, A1B2, A2B1, A3B0, A0B2, A2B0)
                                mma<MODE>(dr, A_(0), B_(0), idesc<MODE>(false, 2 * BN), acc);   // A0 [B1 | B3]
                                mma<MODE>(dr, A_(1), B_(2), idesc<MODE>(false, 2 * BN), 1u);    // A1 [B0 | B2]
                                mma<MODE>(dr, A_(2), B_(1), idesc<MODE>(true), 1u);             // -A2 B3
                                mma<MODE>(di, A_(2), B_(0), idesc<MODE>(false), 1u);            // A2 B1
                                mma<MODE>(dr, A_(3), B_(3), idesc<MODE>(true), 1u);             // -A3 B2
                                mma<MODE>(di, A_(3), B_(2), idesc<MODE>(false), 1u);            // A3 B0
                                mma<MODE>(dr, A_(0), B_(2), idesc<MODE>(false, 2 * BN), 1u);    // A0 [B0 | B2]
                                mma<MODE>(dr, A_(2), B_(3), idesc<MODE>(true), 1u);             // -A2 B2
                                mma<MODE>(di, A_(2), B_(2), idesc<MODE>(false), 1u);            // A2 B0
                            }
                        }
                        mma_commit(&empty_bar[s]);   // frees the stage once these MMAs are done
                    }
                    if (go) mma_commit(&accf[b]);    // chunk gc is complete in accumulator b
                }
            }
            mma_commit(&fin_bar);                    // every MMA of this thread has completed
            mbar_wait(&fin_bar, 0, &abort_flag, false);
        }
    } else {
        // ---------------------------------------------------------- accumulators
        const int e = warp - 2;                 // 0..7
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int h = e >> 2;                   // column half of the tile
        const int r = q * 32 + lane;            // output row of this thread
        const int64_t M = sd.M, N = sd.N;
        // C along n in unit-stride runs of 8 whose offsets (and every offset
        // along m, and the imaginary plane's) are multiples of 4 floats, on a
        // 16-byte boundary: a thread's 64 outputs of its row go out as float4s
        const bool cvec = (sd.flags & kFlagCNVec) && ((uintptr_t)sd.c & 15) == 0 && sd.c_plane % 4 == 0;
        bool ok = true;
        int gc = 0;
        for (int i = 0; i < mytiles && ok; ++i) {
            float sr[64], si[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) sr[j] = si[j] = 0.f;
            for (int c = 0; c < nchunks; ++c, ++gc) {
                const int b = gc & 1;
                ok = mbar_wait(&accf[b], (gc >> 1) & 1, &abort_flag);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 2 * BN + h * 64;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t vr[16], vi[16];
                    tmem_ld16(base + j * 16, vr);
                    tmem_ld16(base + BN + j * 16, vi);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        sr[j * 16 + t] += __uint_as_float(vr[t]);
                        si[j * 16 + t] += __uint_as_float(vi[t]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[b]);   // accumulator b may be overwritten
            }
            if (!ok || abort_flag) break;
            // the tile's sum to C, while the tensor core runs on into the next tile
            int64_t m0, n0;
            tile_origin(first + (int64_t)i * G, m0, n0);
            {
                float *C = (float *)sd.c;
                const int64_t cp = sd.c_plane;
                const bool rok = m0 + r < M;
                const int64_t cm = rok ? sd.offCM[m0 + r] : 0;
                // the warp's 64 column offsets: two coalesced loads, then
                // shuffled to every lane (all lanes take part)
                const int64_t nb = n0 + h * 64;
                const int64_t olo = nb + lane < N ? __ldg(sd.offCN + nb + lane) : 0;
                const int64_t ohi = nb + 32 + lane < N ? __ldg(sd.offCN + nb + 32 + lane) : 0;
                if (cvec) {   // runs of 4 along n: 16-byte stores
#pragma unroll
                    for (int j = 0; j < 64; j += 4) {
                        const int64_t o = cm + __shfl_sync(0xffffffffu, j < 32 ? olo : ohi, j & 31);
                        if (rok && nb + j < N) {
                            *reinterpret_cast<float4 *>(C + o) = make_float4(sr[j], sr[j + 1], sr[j + 2], sr[j + 3]);
                            *reinterpret_cast<float4 *>(C + o + cp) =
                                make_float4(si[j], si[j + 1], si[j + 2], si[j + 3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int64_t o = cm + __shfl_sync(0xffffffffu, j < 32 ? olo : ohi, j & 31);
                        if (rok && nb + j < N) {
                            C[o] = sr[j];
                            C[o + cp] = si[j];
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// 3. plain FP32 products on the CUDA cores from packed operands
// ---------------------------------------------------------------------------
// The FP32 precision: f32_gemm_kernel streams (BM or BN) x BK boxes of each
// operand, viewed as a [2 planes][K][rows] array (rows contiguous), into a
// ring of shared-memory stages with 3-D TMA tensor copies, so the inner loop
// is FFMAs and shared-memory loads only: no per-element address arithmetic,
// no offset-table reads.  An operand already stored that way (a dense K x rows
// matrix in each plane, kFlagADense / kFlagBDense: the network executor lays
// out the intermediates that feed this kernel so) is read in place, the
// index permutation of the step folded into the tensor map; any other layout
// is first gathered once through its offset tables by f32_pack_kernel into a
// padded [2 planes][Kpad][Rpad] workspace.  Each complex product is the four
// real FP32 products of the definition, accumulated in FP32 registers over
// every matched block pair of the tile (Sec. II-C steps 2-4) in a fixed
// order.
namespace f32p {

constexpr int BK = 32;   // k rows of a stage (the tensor maps' box depth)
constexpr int KQ = 32;   // k tile of the pack kernel
constexpr int KU = 2;    // unroll of the two-row inner loop
static_assert(KQ % BK == 0, "k tiles");

// Tile configurations of the GEMM.  A CTA computes a BM x BN complex tile;
// its threads form GY x GX groups of TM x TN outputs (TN adjacent columns),
// and KG such sets split the k rows of every stage between them, their
// partial tiles summed in set order at the end.
template <int BM_, int BN_, int TM_, int TN_, int KG_, int STAGES_>
struct Cfg {
    static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, KG = KG_;
    static constexpr int GX = BN / TN, GY = BM / TM;
    static constexpr int NT = GX * GY * KG;
    static constexpr int STAGES = STAGES_, KR = BK / KG;  // k rows of a stage per set
    static constexpr int PA = BK * BM, PB = BK * BN;      // floats of one plane of one stage
    static constexpr uint32_t STAGE_BYTES = 2u * (PA + PB) * 4u;
    static constexpr size_t RING_BYTES = (size_t)STAGES * STAGE_BYTES;
    static constexpr size_t SMEM = RING_BYTES + 128;
    // a thread's TM rows are consecutive (read as float4), as are its columns
    static_assert(GY * TM == BM && GX * TN == BN && TM % 4 == 0 && TN % 4 == 0 && KR * KG == BK && KR % 2 == 0 &&
                      (GX * GY) % 32 == 0 && BM + BN <= NT,
                  "tile shape");
    static_assert((PA * 4) % 128 == 0 && (PB * 4) % 128 == 0, "stage planes 128-byte aligned (TMA destinations)");
    // a finished C tile is staged as planes of [BN][BM + 4] (or [BM][BN + 4])
    // floats: one at a time through the stage just consumed (mid-stream, one
    // set of threads), or both through the idle ring after a CTA's last unit,
    // behind the other sets' partial tiles ([KG - 1][2 TM TN][GX GY] floats)
    static constexpr size_t PLANE_MAX = (size_t)(BM + 4) * (BN + 4);
    static_assert(KG > 1 || PLANE_MAX * 4 <= STAGE_BYTES, "a staged plane must fit one stage");
    static_assert(((size_t)(KG - 1) * 2 * TM * TN * GX * GY + 2 * PLANE_MAX) * 4 <= RING_BYTES,
                  "the sets' tiles and both staged planes must fit the ring");
};
// One CTA per tile, and stream-K: two sets of 8 x 16 threads of 8 x 4
// outputs, each set half of every stage's k rows.  A thread reads 96 bytes of fragments from
// shared memory per 128 FMAs, where 4 x 4 outputs read 64 per 64 and keep
// shared memory as busy as the FMA pipe: 61.0 against 57.5 TFLOP/s on
// 1024 x 32768 x 1024, 49.3 against 51.2 us on 4096 x 256 x 256.
using Tile8x4 = Cfg<64, 64, 8, 4, 2, 3>;
constexpr int BM = 64, BN = 64;   // its tile (also of the stream-K schedule)
static_assert(Tile8x4::BM == BM && Tile8x4::BN == BN, "tiles");
// Few columns (N <= 16) and a long contraction, e.g. 256 x 16 x 4096: 128 x
// 16 tiles, four sets of 32 x 2 threads of 4 x 8 outputs, the contraction
// split over CTAs (each a run of k-tiles, its partial tile stored and the
// partials summed in split order by f32_split_reduce_kernel): the work is
// too small to fill the SMs with tiles, and each CTA streams its share of
// the large operand once.
using TileSkinny = Cfg<128, 16, 4, 8, 4, 2>;

struct Args {
    CUtensorMap mapA, mapB;   // operands as 3-D {rows, K, 2 planes} FP32 arrays
    GroupArgs g;              // the problem (C pointer, C offset tables, M, N, K, tiles)
    float *sk_part;           // stream-K: partial tiles [tile][piece][2][BM * BN] (fragment order)
    int32_t *sk_count;        // stream-K: pieces stored per tile (0 between launches)
    float *split_part;        // split contraction: partial results [split][2 planes][M x N], row-major (m, n)
    int32_t nkt;              // k-stages (Kpad / BK)
    int32_t sk_maxpieces;     // stream-K: most pieces of any tile
    int32_t sk_dp;            // stream-K: CTAs [0, sk_dp) take tiles [0, sk_dp) whole
};

// out[p][k][r] = operand(r, k) plane p (0 outside R x K), for A (the first
// na CTAs) and then B.  Each CTA packs 32 rows x PKT k, transposed through
// shared memory so that the gather (along the operand's unit-stride digit)
// and the store (along rows) both coalesce; every thread has 16 independent
// loads in flight.
constexpr int PKT = 128;
__global__ void __launch_bounds__(256) f32_pack_kernel(const __grid_constant__ GroupArgs g, float *__restrict__ outA,
                                                       float *__restrict__ outB, int64_t Mpad, int64_t Npad,
                                                       int64_t Kpad, int64_t na, int skip_a) {
    __shared__ GettDesc sd;
    __shared__ float tr[2][PKT][33];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const int which = (skip_a || (int64_t)blockIdx.x >= na) ? 1 : 0;
    const int64_t bid = (int64_t)blockIdx.x - (which && !skip_a ? na : 0);
    const float *__restrict__ src = (const float *)(which ? sd.b : sd.a);
    float *__restrict__ out = which ? outB : outA;
    const int64_t Rpad = which ? Npad : Mpad;
    const int64_t plane = which ? sd.b_plane : sd.a_plane;
    const int64_t *__restrict__ offR = which ? sd.offBN : sd.offAM;
    const int64_t *__restrict__ offK = which ? sd.offBK : sd.offAK;
    const int64_t R = which ? sd.N : sd.M, K = sd.K;
    const bool row_fast = which ? (sd.flags & kFlagBNFast) : (sd.flags & kFlagAMFast);
    const int64_t rtiles = Rpad / 32;
    const int64_t r0 = (bid % rtiles) * 32, k0 = (bid / rtiles) * PKT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    constexpr int NE = 32 * PKT / 256;                        // elements per thread
    int64_t o[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) {   // offsets first (static tables), operands after the wait
        // lanes along rows (row-fast operand) or along k (k-fast operand)
        const int rr = row_fast ? tx : ty + 8 * (j & 3);
        const int kk = row_fast ? ty + 8 * j : tx + 32 * (j >> 2);
        const int64_t r = r0 + rr, k = k0 + kk;
        o[j] = (r < R && k < K) ? offR[r] + offK[k] : -1;
    }
    grid_dep_wait();
    float xr[NE], xi[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        xr[j] = o[j] >= 0 ? src[o[j]] : 0.f;
        xi[j] = o[j] >= 0 ? src[o[j] + plane] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        const int rr = row_fast ? tx : ty + 8 * (j & 3);
        const int kk = row_fast ? ty + 8 * j : tx + 32 * (j >> 2);
        tr[0][kk][rr] = xr[j];
        tr[1][kk][rr] = xi[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        const int kk = ty + 8 * j, rr = tx;
        if (k0 + kk >= Kpad) break;
        const size_t e = (size_t)(k0 + kk) * Rpad + (r0 + rr);
        out[e] = tr[0][kk][rr];
        out[(size_t)Kpad * Rpad + e] = tr[1][kk][rr];
    }
}

// Write a finished tile staged in shared memory to the output (C, or a
// split's partial result) with the lanes of a warp along its unit-stride
// dimension (m if m_fast, else n).  The staged plane holds (BM + 1) x BN
// (m_fast) or BM x (BN + 1) floats, row length ld; `both`: the imaginary
// plane follows at cs + plane, otherwise cs holds plane `pl` alone.  om / on:
// the output offsets of the tile's rows and columns (-1 past M or N), already
// in shared memory, so no store waits on a table load; cp: the output's
// plane stride.
template <class Tile>
__device__ __forceinline__ void emit_tile(const float *cs, int plane, int ld, bool m_fast, bool both, int pl,
                                          const int64_t *om, const int64_t *on, float *base, int64_t cp,
                                          int warp, int lane) {
    constexpr int BM = Tile::BM, BN = Tile::BN, NT = Tile::NT;
    float *out = base + (pl ? cp : 0);
    if (m_fast) {
        int64_t cm[(BM + 31) / 32];
#pragma unroll
        for (int u = 0; u < (BM + 31) / 32; ++u) cm[u] = lane + 32 * u < BM ? om[lane + 32 * u] : -1;
        for (int nl = warp; nl < BN; nl += NT / 32) {
            const int64_t c0 = on[nl];
            if (c0 < 0) break;
#pragma unroll
            for (int u = 0; u < (BM + 31) / 32; ++u)
                if (cm[u] >= 0) {
                    out[cm[u] + c0] = cs[nl * ld + lane + 32 * u];
                    if (both) out[cm[u] + c0 + cp] = cs[plane + nl * ld + lane + 32 * u];
                }
        }
    } else {
        int64_t cn[(BN + 31) / 32];
#pragma unroll
        for (int u = 0; u < (BN + 31) / 32; ++u) cn[u] = lane + 32 * u < BN ? on[lane + 32 * u] : -1;
        for (int ml = warp; ml < BM; ml += NT / 32) {
            const int64_t c0 = om[ml];
            if (c0 < 0) break;
#pragma unroll
            for (int u = 0; u < (BN + 31) / 32; ++u)
                if (cn[u] >= 0) {
                    out[c0 + cn[u]] = cs[ml * ld + lane + 32 * u];
                    if (both) out[c0 + cn[u] + cp] = cs[plane + ml * ld + lane + 32 * u];
                }
        }
    }
}

// CTA index owning unit u when U units are split evenly over G CTAs (CTA c
// takes units [c U / G, (c + 1) U / G)).
__device__ __forceinline__ int64_t sk_owner(int64_t u, int64_t U, int64_t G) { return ((u + 1) * G - 1) / U; }

// Work is a sequence of units (output tile t, k-tile kt), k fastest.  Without
// kFlagStreamK a CTA takes the units of one tile (data-parallel).  With it
// (stream-K) the launch has G CTAs: the first D = sk_dp take tiles [0, D)
// whole, and CTA D + c takes units [c U' / G', (c + 1) U' / G') of the U' =
// (tiles - D) * nkt units of the other tiles, G' = G - D, so that every SM
// gets the same work however the tile count divides the SMs (D = SMs when
// the tiles number between one and two per SM: each SM holds one whole tile
// and a share of the rest).  A CTA holding only part of a tile's k range
// writes that partial tile to the workspace and counts it in the tile's
// counter; the CTA that brings the count to the number of pieces sums the
// pieces in k order (a fixed order: results do not depend on scheduling),
// writes C and resets the counter.  No CTA ever waits for another.
template <class C, bool SK>
__global__ void __launch_bounds__(C::NT, 2) f32_gemm_kernel(const __grid_constant__ Args p) {
    constexpr int NT = C::NT, BM = C::BM, BN = C::BN, TM = C::TM, TN = C::TN, STAGES = C::STAGES;
    constexpr int PA = C::PA, PB = C::PB, GX = C::GX, GY = C::GY, KR = C::KR;
    constexpr uint32_t STAGE_BYTES = C::STAGE_BYTES;
    constexpr int GXY = GX * GY, FV = 2 * TM * TN;   // threads of a set, values a thread holds
    // stream-K stages a tile's sets and then one C plane at a time through a
    // single consumed stage
    static_assert(!SK || ((size_t)FV * GXY * 4 <= STAGE_BYTES && C::PLANE_MAX * 4 <= STAGE_BYTES), "stage size");
    extern __shared__ unsigned char dsm_raw[];
    float *stg = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~(uintptr_t)127);
    __shared__ GettDesc sd;
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ volatile int abort_flag;
    __shared__ int last_piece;
    __shared__ int64_t c_om[BM], c_on[BN];   // output offsets of the current tile's rows and columns
    __shared__ int64_t cta_u0, cta_u1;   // this CTA's unit range (stream-K; out of the k loop's registers)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    grid_dep_launch();
    if (warp == 0) load_desc(p.g, sd);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full_bar[s], 1);
            tc::mbar_init(&empty_bar[s], NT / 32);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nkt = p.nkt;
    // raster: the operand with fewer tiles varies fastest (its tiles stay in L2)
    const bool n_fast = sd.tiles_n < sd.tiles_m;
    auto tile_origin = [&](int64_t t, int &m0, int &n0) {
        const int64_t tm = n_fast ? t / sd.tiles_n : t % sd.tiles_m;
        const int64_t tn = n_fast ? t % sd.tiles_n : t / sd.tiles_m;
        m0 = (int)(tm * BM);
        n0 = (int)(tn * BN);
    };
    // stream-K: whole tiles for CTAs [0, D), the units of tiles [D, tiles)
    // split evenly over the other Gs CTAs; owner(u): the CTA holding unit u
    auto owner = [&](int64_t u) {
        const int64_t D = p.sk_dp, ub = D * nkt;
        const int64_t Us = sd.tiles_m * sd.tiles_n * (int64_t)nkt - ub, Gs = (int64_t)gridDim.x - D;
        return u < ub ? u / nkt : D + sk_owner(u - ub, Us, Gs);
    };
    // one tile per CTA, or with a split contraction (ksplit > 1) CTA
    // (tile, split) takes k-tiles [split kps, (split + 1) kps) of its tile and
    // stores a partial result
    const int ksplit = SK ? 1 : max(1, sd.ksplit);
    int split = 0;
    int64_t u0, u1;
    if (SK) {
        const int64_t D = p.sk_dp, ub = D * nkt;
        const int64_t Us = sd.tiles_m * sd.tiles_n * (int64_t)nkt - ub, Gs = (int64_t)gridDim.x - D;
        const int64_t c = (int64_t)blockIdx.x - D;
        u0 = c < 0 ? (int64_t)blockIdx.x * nkt : ub + c * Us / Gs;
        u1 = c < 0 ? u0 + nkt : ub + (c + 1) * Us / Gs;
    } else {
        const int64_t cta = (int64_t)blockIdx.x - sd.tile_begin;
        split = (int)(cta % ksplit);
        const int kt0 = ksplit > 1 ? split * sd.ktiles_per_split : 0;
        const int kt1 = ksplit > 1 ? min(nkt, kt0 + sd.ktiles_per_split) : nkt;
        u0 = (cta / ksplit) * nkt + kt0;
        u1 = (cta / ksplit) * nkt + kt1;
    }
    const int nitems = (int)(u1 - u0);
    if (tid == 0) {   // the tensor maps into the TMA unit's cache while the previous kernel ends
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.mapB)) : "memory");
    }
    grid_dep_wait();   // operands may be the previous kernel's output
    // the output offsets of a tile's rows and columns into shared memory, one
    // per thread (-1 past M or N): C's, or the row-major (m, n) of a partial
    auto load_offsets = [&](int m0, int n0) {
        if (tid < BM) {
            const int64_t m = m0 + tid;
            c_om[tid] = m >= sd.M ? -1 : ksplit > 1 ? m * sd.N : __ldg(sd.offCM + m);
        } else if (tid < BM + BN) {
            const int64_t n = n0 + tid - BM;
            c_on[tid - BM] = n >= sd.N ? -1 : ksplit > 1 ? n : __ldg(sd.offCN + n);
        }
    };

    // units are issued (one thread) and consumed strictly in order: each side
    // walks (tile, k-tile) with its own cursor instead of dividing per unit
    int pt = (int)(u0 / nkt);   // producer cursor (stream-K): tile, k-tile, tile origin
    int pkt = (int)(u0 % nkt), pm0 = 0, pn0 = 0;
    tile_origin(pt, pm0, pn0);
    auto issue = [&](int i) {   // one thread: the next unit (u0 + i) into its stage
        const int s = i % STAGES;
        const int kt = SK ? pkt : pkt + i;   // one tile per CTA: unit i is k-tile pkt + i
        tc::mbar_expect_tx(&full_bar[s], STAGE_BYTES);
        const uint32_t sa = tc::su32(stg + (size_t)s * 2 * (PA + PB));
        const uint32_t sb = sa + 2u * PA * 4u;
        tc::tma_load_3d(sa, &p.mapA, pm0, kt * BK, 0, &full_bar[s]);
        tc::tma_load_3d(sa + PA * 4u, &p.mapA, pm0, kt * BK, 1, &full_bar[s]);
        tc::tma_load_3d(sb, &p.mapB, pn0, kt * BK, 0, &full_bar[s]);
        tc::tma_load_3d(sb + PB * 4u, &p.mapB, pn0, kt * BK, 1, &full_bar[s]);
        if (SK && ++pkt == nkt) {
            pkt = 0;
            tile_origin(++pt, pm0, pn0);
        }
    };
    int issued = 0;
    if (tid == 0) {
        if (SK) {
            cta_u0 = u0;
            cta_u1 = u1;
        }
        for (; issued < min(STAGES, nitems); ++issued) issue(issued);
    }
    // one tile per CTA: its offsets load while the first stages land (the
    // barriers before the epilogue's stores publish them)
    if (!SK) load_offsets(pm0, pn0);
    int ct = (int)(u0 / nkt);   // consumer cursor
    int ckt = (int)(u0 % nkt);

    const int tx = tid % GX, ty = (tid / GX) % GY, kg = tid / (GX * GY);   // column group, row group, k set
    float cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0.f;

    auto frag = [&](const float *a0, const float *b0, int kk, float *xr, float *xi, float *yr, float *yi) {
#pragma unroll
        for (int v = 0; v < TM / 4; ++v) {
            const float4 r = *reinterpret_cast<const float4 *>(a0 + kk * BM + 4 * v);
            const float4 q = *reinterpret_cast<const float4 *>(a0 + PA + kk * BM + 4 * v);
            xr[4 * v] = r.x; xr[4 * v + 1] = r.y; xr[4 * v + 2] = r.z; xr[4 * v + 3] = r.w;
            xi[4 * v] = q.x; xi[4 * v + 1] = q.y; xi[4 * v + 2] = q.z; xi[4 * v + 3] = q.w;
        }
#pragma unroll
        for (int v = 0; v < TN / 4; ++v) {
            const float4 r = *reinterpret_cast<const float4 *>(b0 + kk * BN + 4 * v);
            const float4 q = *reinterpret_cast<const float4 *>(b0 + PB + kk * BN + 4 * v);
            yr[4 * v] = r.x; yr[4 * v + 1] = r.y; yr[4 * v + 2] = r.z; yr[4 * v + 3] = r.w;
            yi[4 * v] = q.x; yi[4 * v + 1] = q.y; yi[4 * v + 2] = q.z; yi[4 * v + 3] = q.w;
        }
    };
    // the complex products of one k row, two adjacent output columns per
    // packed two-wide FMA: B's real and imaginary rows give the column pairs
    // as loaded, A's entries are duplicated into pairs.  The same FMAs in the
    // same order as four scalar FMAs per product (bitwise equal results) in
    // half the issue slots (57.4 against 55.8 TFLOP/s on 1024 x 32768 x 1024).
    // A's real parts go out for every row before its imaginary parts, so the
    // two FMAs into one accumulator pair are a row pass apart instead of
    // adjacent (4096 x 256 x 256: 49.4 -> 47.5 us; each accumulator's order
    // unchanged)
    auto macs = [&](const float *xr, const float *xi, const float *yr, const float *yi) {
        float2 br2[TN / 2], bi2[TN / 2], nbi2[TN / 2];
#pragma unroll
        for (int jp = 0; jp < TN / 2; ++jp) {
            br2[jp] = make_float2(yr[2 * jp], yr[2 * jp + 1]);
            bi2[jp] = make_float2(yi[2 * jp], yi[2 * jp + 1]);
            nbi2[jp] = make_float2(-yi[2 * jp], -yi[2 * jp + 1]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {   // the real parts of A first, for every row
            const float2 ar2 = make_float2(xr[i], xr[i]);
#pragma unroll
            for (int jp = 0; jp < TN / 2; ++jp) {
                float2 r = make_float2(cr[i][2 * jp], cr[i][2 * jp + 1]);
                float2 q = make_float2(ci[i][2 * jp], ci[i][2 * jp + 1]);
                r = __ffma2_rn(ar2, br2[jp], r);
                q = __ffma2_rn(ar2, bi2[jp], q);
                cr[i][2 * jp] = r.x; cr[i][2 * jp + 1] = r.y;
                ci[i][2 * jp] = q.x; ci[i][2 * jp + 1] = q.y;
            }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {   // then the imaginary parts
            const float2 ai2 = make_float2(xi[i], xi[i]);
#pragma unroll
            for (int jp = 0; jp < TN / 2; ++jp) {
                float2 r = make_float2(cr[i][2 * jp], cr[i][2 * jp + 1]);
                float2 q = make_float2(ci[i][2 * jp], ci[i][2 * jp + 1]);
                r = __ffma2_rn(ai2, nbi2[jp], r);
                q = __ffma2_rn(ai2, br2[jp], q);
                cr[i][2 * jp] = r.x; cr[i][2 * jp + 1] = r.y;
                ci[i][2 * jp] = q.x; ci[i][2 * jp + 1] = q.y;
            }
        }
    };

    // Several k sets hold partial tiles of the same outputs: sets 1, 2, ...
    // store theirs in fragment order through `scratch` (FV x GXY floats a set
    // after the first; consecutive threads, consecutive words: no bank
    // conflicts) and set 0 adds them in set order, ((s0 + s1) + s2) + ...,
    // the same in every CTA.  Set 0 then holds the tile.
    auto merge_sets = [&](float *scratch) {
        if constexpr (C::KG > 1) {
            const int tin = tid % GXY;
            __syncthreads();   // the scratch area is free
            if (kg > 0) {
                float *f = scratch + (size_t)(kg - 1) * FV * GXY + tin;
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        f[(i * TN + j) * GXY] = cr[i][j];
                        f[(TM * TN + i * TN + j) * GXY] = ci[i][j];
                    }
            }
            __syncthreads();
            if (kg == 0) {
#pragma unroll 1
                for (int g = 1; g < C::KG; ++g) {
                    const float *f = scratch + (size_t)(g - 1) * FV * GXY + tin;
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) {
                            cr[i][j] += f[(i * TN + j) * GXY];
                            ci[i][j] += f[(TM * TN + i * TN + j) * GXY];
                        }
                }
            }
        }
    };

    // the finished tile at (m0, n0), its sets merged first unless `merged`.
    // `cs`: a consumed stage (mid-stream), which serves the merge and then
    // stages one plane at a time, or the whole idle ring after the CTA's last
    // unit (the merge, then both planes behind it).  A split's partial result
    // goes straight to global memory (row-major (m, n), n fastest); C is
    // staged through shared memory as [BN][BM + 4] (or [BM][BN + 4]) planes
    // written as float4 by set 0 and stored with the lanes of a warp along
    // C's unit-stride dimension (m unless kFlagCNFast).
    auto store_c = [&](float *cs, bool both, int m0, int n0, bool merged) {
        if (SK) {   // this tile's offsets (the previous tile's stores are done)
            __syncthreads();
            load_offsets(m0, n0);
        }
        if (!merged) merge_sets(cs);
        float *stage = both ? cs + (C::KG - 1) * FV * GXY : cs;
        if (ksplit > 1) {   // this split's partial result, from set 0's registers
            if (kg != 0) return;
            const int64_t M = sd.M, N = sd.N, MN = M * N;
            float *out = p.split_part + 2 * (int64_t)split * MN;
            const bool vec = (N & 3) == 0;
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const int64_t m = m0 + ty * TM + i;
                if (m >= M) break;
#pragma unroll
                for (int v = 0; v < TN / 4; ++v) {
                    const int64_t n = n0 + tx * TN + 4 * v;
                    float *o = out + m * N + n;
                    if (vec && n + 3 < N) {
                        *reinterpret_cast<float4 *>(o) =
                            make_float4(cr[i][4 * v], cr[i][4 * v + 1], cr[i][4 * v + 2], cr[i][4 * v + 3]);
                        *reinterpret_cast<float4 *>(o + MN) =
                            make_float4(ci[i][4 * v], ci[i][4 * v + 1], ci[i][4 * v + 2], ci[i][4 * v + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (n + e < N) {
                                o[e] = cr[i][4 * v + e];
                                o[e + MN] = ci[i][4 * v + e];
                            }
                    }
                }
            }
            return;
        }
        const bool m_fast = !(sd.flags & kFlagCNFast);
        const int ld = m_fast ? BM + 4 : BN + 4;   // row length of a staged plane (float4-aligned)
        const int plane = (m_fast ? BN : BM) * ld;
        auto put = [&](float *dst, const float (*x)[TN]) {
            if (m_fast) {
#pragma unroll
                for (int j = 0; j < TN; ++j)
#pragma unroll
                    for (int v = 0; v < TM / 4; ++v)
                        *reinterpret_cast<float4 *>(dst + (tx * TN + j) * ld + ty * TM + 4 * v) =
                            make_float4(x[4 * v][j], x[4 * v + 1][j], x[4 * v + 2][j], x[4 * v + 3][j]);
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int v = 0; v < TN / 4; ++v)
                        *reinterpret_cast<float4 *>(dst + (ty * TM + i) * ld + tx * TN + 4 * v) =
                            make_float4(x[i][4 * v], x[i][4 * v + 1], x[i][4 * v + 2], x[i][4 * v + 3]);
            }
        };
#pragma unroll 1
        for (int pl = 0; pl < (both ? 1 : 2); ++pl) {
            __syncthreads();   // the staging area is free
            if (kg == 0) {
                if (both) {
                    put(stage, cr);
                    put(stage + plane, ci);
                } else {
                    put(stage, pl ? ci : cr);
                }
            }
            __syncthreads();
            emit_tile<C>(stage, plane, ld, m_fast, both, pl, c_om, c_on, (float *)sd.c, sd.c_plane, warp, lane);
        }
        __syncthreads();   // the staging area may be refilled
    };

    int done0 = 0;   // units whose full barrier thread 0 has passed
    for (int i = 0; i < nitems; ++i) {
        const int s = i % STAGES;
        // every lane observes the phase itself; the warp leaves together
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_fast(&full_bar[s], (i / STAGES) & 1, &abort_flag));
        if (!ok) break;
        if (tid == 0) done0 = i + 1;
        // this thread's rows and columns in the stage, from its set's first k row
        const float *a0 = stg + (size_t)s * 2 * (PA + PB) + kg * KR * BM + ty * TM;
        const float *b0 = stg + (size_t)s * 2 * (PA + PB) + 2 * PA + kg * KR * BN + tx * TN;
        float xr0[TM], xi0[TM], yr0[TN], yi0[TN];
        if constexpr (C::TM * C::TN <= 16) {   // the next row's fragments load while this row's FMAs run
            float xr1[TM], xi1[TM], yr1[TN], yi1[TN];
            frag(a0, b0, 0, xr0, xi0, yr0, yi0);
#pragma unroll(KU)
            for (int kk = 0; kk < KR - 2; kk += 2) {
                frag(a0, b0, kk + 1, xr1, xi1, yr1, yi1);
                macs(xr0, xi0, yr0, yi0);
                frag(a0, b0, kk + 2, xr0, xi0, yr0, yi0);
                macs(xr1, xi1, yr1, yi1);
            }
            frag(a0, b0, KR - 1, xr1, xi1, yr1, yi1);   // last two rows: no prefetch
            macs(xr0, xi0, yr0, yi0);
            macs(xr1, xi1, yr1, yi1);
        } else {   // more outputs a thread: no registers for a second set of fragments
            // 8 x 4 outputs: unrolled 8 (62.6 against 61.8 TFLOP/s with 4 on
            // 1024 x 32768 x 1024); 4 x 8 outputs spill when unrolled past 4
            constexpr int KU1 = C::TM == 8 ? 8 : 4;
#pragma unroll(KU1)
            for (int kk = 0; kk < KR; ++kk) {
                frag(a0, b0, kk, xr0, xi0, yr0, yi0);
                macs(xr0, xi0, yr0, yi0);
            }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty_bar[s]);
        // warp 0 refills the stage consumed one unit ago (all warps have
        // normally released it by now), keeping STAGES - 1 units ahead; the
        // whole warp takes the branch so that no lane computes alone
        if (warp == 0 && i >= 1 && i - 1 + STAGES < nitems) {
            bool ok2 = true;
            if (lane == 0) {
                const int t = i - 1;
                ok2 = tc::mbar_wait_fast(&empty_bar[t % STAGES], (t / STAGES) & 1, &abort_flag);
                if (ok2) {
                    issue(t + STAGES);
                    issued = t + STAGES + 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok2 ? 1 : 0, 0)) break;
        }
        if (!SK) continue;   // one tile per CTA: its epilogue follows the loop
        const int t = ct;
        const bool tile_end = ckt == nkt - 1 || i == nitems - 1;
        if (++ckt == nkt) {
            ckt = 0;
            ++ct;
        }
        if (!tile_end) continue;
        // ---- this CTA's range of tile t ends here
        int m0, n0;
        tile_origin(t, m0, n0);
        // stage s holds consumed data and is refilled only after this
        // epilogue (by the next unit's refill): it serves as staging area
        float *cs = stg + (size_t)s * 2 * (PA + PB);
        bool write_c = true, merged = false;
        const int64_t tb = (int64_t)t * nkt;   // the tile's first unit
        if (SK && (cta_u0 > tb || cta_u1 < tb + nkt)) {
            // a piece of the tile: store it (set 0, after the sets are
            // merged), count it, and sum all pieces if it is the last one to
            // arrive
            const int64_t cf = owner(tb);
            const int npieces = (int)(owner(tb + nkt - 1) - cf + 1);
            const int piece = (int)((int64_t)blockIdx.x - cf);
            const int tin = tid % GXY;
            float *slot = p.sk_part + ((int64_t)t * p.sk_maxpieces + piece) * (2 * BM * BN);
            merge_sets(cs);
            merged = true;
            if (kg == 0) {
#pragma unroll
                for (int i2 = 0; i2 < TM; ++i2)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        slot[(i2 * TN + j) * GXY + tin] = cr[i2][j];
                        slot[(TM * TN + i2 * TN + j) * GXY + tin] = ci[i2][j];
                    }
            }
            // the barrier orders every thread's stores before thread 0's
            // release; its acquire orders the other pieces' stores before the
            // barrier after which set 0 reads them
            __syncthreads();
            if (tid == 0) {
                int old;
                asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], 1;" : "=r"(old) : "l"(p.sk_count + t)
                             : "memory");
                last_piece = old == npieces - 1;
            }
            __syncthreads();
            write_c = last_piece;
            if (write_c) {
                if (kg == 0) {
                    const float *base = p.sk_part + (int64_t)t * p.sk_maxpieces * (2 * BM * BN);
#pragma unroll
                    for (int i2 = 0; i2 < TM; ++i2)
#pragma unroll
                        for (int j = 0; j < TN; ++j) cr[i2][j] = ci[i2][j] = 0.f;
                    for (int q = 0; q < npieces; ++q) {   // pieces in k order
                        const float *src = base + (int64_t)q * (2 * BM * BN) + tin;
#pragma unroll
                        for (int i2 = 0; i2 < TM; ++i2)
#pragma unroll
                            for (int j = 0; j < TN; ++j) {
                                cr[i2][j] += __ldcg(src + (i2 * TN + j) * GXY);
                                ci[i2][j] += __ldcg(src + (TM * TN + i2 * TN + j) * GXY);
                            }
                    }
                }
                if (tid == 0) p.sk_count[t] = 0;   // ready for the next launch
            }
        }
        if (write_c) {
            // after the CTA's last unit no copy is in flight: the whole ring
            // stages both planes at once
            if (i == nitems - 1) store_c(stg, true, m0, n0, merged);
            else store_c(cs, false, m0, n0, merged);
        }
#pragma unroll
        for (int i2 = 0; i2 < TM; ++i2)
#pragma unroll
            for (int j = 0; j < TN; ++j) cr[i2][j] = ci[i2][j] = 0.f;
    }
    if (tid == 0)   // no copy may still be landing in shared memory when the CTA exits
        for (int t = done0; t < issued; ++t)
            tc::mbar_wait(&full_bar[t % STAGES], (t / STAGES) & 1, &abort_flag, false);
    __syncthreads();
    if (!SK && !abort_flag) store_c(stg, true, pm0, pn0, false);   // the CTA's tile; the idle ring stages both planes
}

// Sum of the partial results of a split contraction into C, in split order
// (deterministic): 32 outputs per CTA; warp w adds partials w, w + 8, ... of
// its lane's output, then warp 0 adds the eight sums in warp order.  The
// descriptor and C's offsets are read before the wait for the GEMM (planner
// tables, complete before the GEMM started); the partials, which the GEMM
// has just written, after it and through L2.
__global__ void __launch_bounds__(256) f32_split_reduce_kernel(const __grid_constant__ GroupArgs g,
                                                               const float *__restrict__ part, int nsplit) {
    __shared__ GettDesc sd;
    __shared__ float red[2][8][33];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const int64_t MN = sd.M * sd.N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t o = ((int64_t)blockIdx.x - sd.tile_begin) * 32 + lane;
    int64_t ic = -1;
    if (w == 0 && o < MN) ic = __ldg(sd.offCM + o / sd.N) + __ldg(sd.offCN + o % sd.N);
    grid_dep_wait();
    float sr = 0.f, si = 0.f;
    if (o < MN) {
#pragma unroll 4
        for (int sp = w; sp < nsplit; sp += 8) {
            sr += __ldcg(part + (2 * (int64_t)sp) * MN + o);
            si += __ldcg(part + (2 * (int64_t)sp + 1) * MN + o);
        }
    }
    red[0][w][lane] = sr;
    red[1][w][lane] = si;
    __syncthreads();
    if (w != 0 || o >= MN) return;
    sr = red[0][0][lane];
    si = red[1][0][lane];
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        sr += red[0][j][lane];
        si += red[1][j][lane];
    }
    float *C = (float *)sd.c;
    C[ic] = sr;
    C[ic + sd.c_plane] = si;
}

}  // namespace f32p

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

int tc_tile_m() { return tc::BM; }
int tc_tile_n() { return tc::BN; }

namespace {

struct TcGeom {
    int esz, bk, narr, narr_b;
    int64_t Mpad, Npad, Kpad;
    size_t arrA, arrB;   // bytes of one packed array
};

TcGeom tc_geom(const GettDesc &d, int mode) {
    TcGeom g;
    g.esz = mode == tc::kBF16x3 ? 2 : 4;
    g.bk = tc::ROWB / g.esz;
    g.narr = mode == tc::kTF32 ? 2 : 4;
    g.narr_b = mode == tc::kTF32 ? 3 : 4;
    g.Mpad = (d.M + tc::BM - 1) / tc::BM * tc::BM;
    g.Npad = (d.N + tc::BN - 1) / tc::BN * tc::BN;
    const int64_t kq = 32;   // the pack kernel's k tile; a multiple of bk
    g.Kpad = (d.K + kq - 1) / kq * kq;
    g.arrA = (size_t)g.Mpad * g.Kpad * g.esz;
    g.arrB = (size_t)g.Npad * g.Kpad * g.esz;
    return g;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    if (!fn) RN_FAIL(ROSNET_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    return fn;
}

// 2-D map over one packed [rows][Kpad] array, boxes of (64 bytes of k) x 128 rows.
void make_map(CUtensorMap *m, void *base, int64_t rows, int64_t Kpad, int esz) {
    cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(Kpad * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(tc::ROWB / esz), 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                             2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) RN_FAIL(ROSNET_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

template <int MODE>
void launch_mode(const GroupArgs &ga, const TcGeom &g, void *ws, int64_t ctas, cudaStream_t s,
                 bool pack_a, bool pack_b, const std::function<void()> &before_gemm) {
    using C_ = tc::Cfg<MODE>;
    static std::atomic<uint64_t> done{0};   // once per device
    uint64_t bit;
    if (!attrs_set(done, &bit)) {
        RN_CHECK_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_::SMEM));
        done.fetch_or(bit, std::memory_order_release);
    }
    unsigned char *pa = (unsigned char *)ws;
    unsigned char *pb = pa + g.narr * g.arrA;
    const int64_t ca = (g.Mpad / 32) * (g.Kpad / 32), cb = (g.Npad / 32) * (g.Kpad / 32);
    if (ca > 0x7fffffffLL || cb > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "operand too large to pack");
    if (pack_a) {
        tc::tc_pack_kernel<MODE><<<(unsigned)ca, 256, 0, s>>>(ga, 0, pa, g.Mpad, g.Kpad);
        g_launches++;
    }
    if (pack_b) {
        tc::tc_pack_kernel<MODE><<<(unsigned)cb, 256, 0, s>>>(ga, 1, pb, g.Npad, g.Kpad);
        g_launches++;
    }
    tc::TcArgs args;
    memset(&args, 0, sizeof(args));
    for (int a = 0; a < g.narr; ++a) make_map(&args.mapA[a], pa + a * g.arrA, g.Mpad, g.Kpad, g.esz);
    for (int a = 0; a < g.narr_b; ++a) make_map(&args.mapB[a], pb + a * g.arrB, g.Npad, g.Kpad, g.esz);
    args.g = ga;
    args.nkt = (int)(g.Kpad / g.bk);
    if (before_gemm) before_gemm();
    // persistent: one CTA per SM (its shared memory allows no second one)
    const int64_t grid = std::min<int64_t>(ctas, (int64_t)num_sms());
    tc::tc_gemm_kernel<MODE><<<(unsigned)grid, tc::NTHREADS, C_::SMEM, s>>>(args);
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

// The GEMM's workspace: [stream-K tile counters | stream-K partial tiles |
// partial results of a split contraction | packed A and B panels], each part
// 256-byte aligned.  The counters, pieces and partials sit at offsets that do
// not depend on the panels, which are left out when both operands are read
// in place.
struct F32Geom {
    int bm, bn;                    // the tile
    int64_t Mpad, Npad, Kpad;
    size_t pack_bytes;             // packed A and B panels
    size_t split_bytes = 0;        // partial results of a split contraction
    // stream-K: CTAs, whole-tile CTAs, split units, most pieces of a tile, and
    // the bytes of the partial tiles and per-tile counters
    int64_t G = 0, D = 0, U = 0, maxpieces = 0;
    size_t part_bytes = 0, count_bytes = 0;
    size_t off_part = 0, off_split = 0, off_pack = 0, total = 0;
};

int64_t sk_owner_host(int64_t u, int64_t U, int64_t G) { return ((u + 1) * G - 1) / U; }

// The GEMM's tile for an M x N output: 128 x 16 for N <= 16, else 64 x 64.
bool f32p_skinny(int64_t N) { return N <= f32p::TileSkinny::BN; }

F32Geom f32_geom(const GettDesc &d, bool both_in_place = false) {
    F32Geom g;
    const bool skinny = f32p_skinny(d.N);
    g.bm = skinny ? f32p::TileSkinny::BM : f32p::BM;
    g.bn = skinny ? f32p::TileSkinny::BN : f32p::BN;
    // panels: rows padded to the tile and to the pack kernel's 32-row tile
    const int64_t rn = std::max(g.bn, 32);
    g.Mpad = (d.M + g.bm - 1) / g.bm * g.bm;
    g.Npad = (d.N + rn - 1) / rn * rn;
    g.Kpad = (d.K + f32p::KQ - 1) / f32p::KQ * f32p::KQ;   // KQ is a multiple of BK
    g.pack_bytes = both_in_place ? 0 : (size_t)2 * (g.Mpad + g.Npad) * g.Kpad * 4;
    if (d.flags & kFlagStreamK) {
        // between one and two tiles per SM: one whole tile per SM, the rest
        // split evenly over a second CTA per SM; otherwise all tiles split
        const int64_t tiles = d.tiles_m * d.tiles_n, nkt = g.Kpad / f32p::BK, sms = num_sms();
        g.D = tiles > sms && tiles < 2 * sms ? sms : 0;
        g.U = (tiles - g.D) * nkt;   // the split units
        g.G = g.D + std::min<int64_t>(g.D ? sms : 2 * sms, g.U);
        const int64_t gs = g.G - g.D;
        for (int64_t t = g.D; t < tiles; ++t)
            g.maxpieces = std::max(g.maxpieces, sk_owner_host((t + 1 - g.D) * nkt - 1, g.U, gs) -
                                                    sk_owner_host((t - g.D) * nkt, g.U, gs) + 1);
        g.part_bytes = (size_t)tiles * g.maxpieces * 2 * f32p::BM * f32p::BN * 4;
        g.count_bytes = ((size_t)tiles * 4 + 255) & ~(size_t)255;
    }
    if (d.ksplit > 1) g.split_bytes = ((size_t)d.ksplit * 2 * (size_t)(d.M * d.N) * 4 + 255) & ~(size_t)255;
    g.off_part = g.count_bytes;
    g.off_split = g.off_part + g.part_bytes;
    g.off_pack = g.off_split + g.split_bytes;
    g.total = g.off_pack + g.pack_bytes;
    return g;
}

// 3-D map over one FP32 operand viewed as [2 planes][K][rows]: {rows, K, 2}
// with the given row and plane strides (elements), boxes of `box_rows` rows x
// BK k x 1 plane (no swizzle: the GEMM reads rows as float4).  Boxes reaching
// past rows or K are filled with zeros.
void make_map_f32(CUtensorMap *m, const void *base, int64_t rows, int64_t K, int64_t row_stride,
                  int64_t plane_stride, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)rows, (cuuint64_t)K, 2};
    cuuint64_t strides[2] = {(cuuint64_t)(row_stride * 4), (cuuint64_t)(plane_stride * 4)};
    cuuint32_t box[3] = {(cuuint32_t)box_rows, (cuuint32_t)f32p::BK, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) RN_FAIL(ROSNET_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

// Whether an operand flagged dense can be read in place by a TMA map: its
// planes start on 16-byte boundaries and its row and plane strides are
// multiples of 16 bytes (every other limit is far above these sizes).
bool tma_direct_ok(bool dense, const void *p, int64_t rows, int64_t K, int64_t plane) {
    return dense && p != nullptr && ((uintptr_t)p & 15) == 0 && rows % 4 == 0 && plane % 4 == 0 &&
           rows < (int64_t(1) << 31) && K < (int64_t(1) << 31) && plane < (int64_t(1) << 37);
}

void launch_f32(const GroupArgs &ga, const GettDesc &d, void *ws, int64_t ctas, cudaStream_t s, bool pack_a,
                bool pack_b, const std::function<void()> &before_gemm, bool pdl) {
    using f32p::Tile8x4;
    using f32p::TileSkinny;
    static std::atomic<uint64_t> done{0};   // once per device
    uint64_t bit;
    if (!attrs_set(done, &bit)) {
        RN_CHECK_CUDA(cudaFuncSetAttribute(f32p::f32_gemm_kernel<Tile8x4, false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile8x4::SMEM));
        RN_CHECK_CUDA(cudaFuncSetAttribute(f32p::f32_gemm_kernel<Tile8x4, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile8x4::SMEM));
        RN_CHECK_CUDA(cudaFuncSetAttribute(f32p::f32_gemm_kernel<TileSkinny, false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TileSkinny::SMEM));
        done.fetch_or(bit, std::memory_order_release);
    }
    // operands stored as dense K x rows matrices are read in place; the others
    // are packed (unless the caller says the workspace already holds them)
    const bool da = tma_direct_ok(d.flags & kFlagADense, d.a, d.M, d.K, d.a_plane);
    const bool db = tma_direct_ok(d.flags & kFlagBDense, d.b, d.N, d.K, d.b_plane);
    const F32Geom g = f32_geom(d, da && db);
    const bool skinny = f32p_skinny(d.N), sk = d.flags & kFlagStreamK, split = d.ksplit > 1;
    if (sk && (skinny || split)) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "stream-K takes 64 x 64 tiles and no split");
    if (split && (d.ktiles_per_split < 1 || (int64_t)d.ksplit * d.ktiles_per_split < g.Kpad / f32p::BK))
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "split does not cover the contraction");
    float *pa = (float *)((char *)ws + g.off_pack);
    float *pb = pa + 2 * g.Mpad * g.Kpad;
    pack_a = pack_a && !da;
    pack_b = pack_b && !db;
    const int64_t kt = (g.Kpad + f32p::PKT - 1) / f32p::PKT;
    const int64_t ca = (g.Mpad / 32) * kt, cb = (g.Npad / 32) * kt;
    if (ca > 0x7fffffffLL || cb > 0x7fffffffLL || 2 * g.Kpad > 0x7fffffffLL || g.Mpad > 0x7fffffffLL ||
        g.Npad > 0x7fffffffLL)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "operand too large to pack");
    if (pack_a || pack_b) {
        const int64_t n = (pack_a ? ca : 0) + (pack_b ? cb : 0);
        if (n > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "operands too large to pack");
        launch_pdl(f32p::f32_pack_kernel, dim3((unsigned)n), 256, 0, s, pdl, ga, pa, pb, g.Mpad, g.Npad, g.Kpad,
                   pack_a ? ca : (int64_t)0, pack_a ? 0 : 1);
        g_launches++;
    }
    f32p::Args args;
    memset(&args, 0, sizeof(args));
    if (da) make_map_f32(&args.mapA, d.a, d.M, d.K, d.M, d.a_plane, g.bm);
    else make_map_f32(&args.mapA, pa, g.Mpad, g.Kpad, g.Mpad, g.Mpad * g.Kpad, g.bm);
    if (db) make_map_f32(&args.mapB, d.b, d.N, d.K, d.N, d.b_plane, g.bn);
    else make_map_f32(&args.mapB, pb, g.Npad, g.Kpad, g.Npad, g.Npad * g.Kpad, g.bn);
    args.g = ga;
    args.nkt = (int)(g.Kpad / f32p::BK);
    if (d.flags & kFlagStreamK) {
        args.sk_part = (float *)((char *)ws + g.off_part);
        args.sk_count = (int32_t *)ws;
        args.sk_maxpieces = (int32_t)g.maxpieces;
        args.sk_dp = (int32_t)g.D;
        ctas = g.G;
    }
    if (split) args.split_part = (float *)((char *)ws + g.off_split);
    if (before_gemm) before_gemm();
    // after a pack the GEMM's prologue may overlap it (it reads only its
    // descriptor before waiting); with no pack it is the first launch
    const bool pdl_gemm = pdl || pack_a || pack_b;
    if (sk)
        launch_pdl(f32p::f32_gemm_kernel<Tile8x4, true>, dim3((unsigned)ctas), Tile8x4::NT, Tile8x4::SMEM, s,
                   pdl_gemm, args);
    else if (skinny)
        launch_pdl(f32p::f32_gemm_kernel<TileSkinny, false>, dim3((unsigned)ctas), TileSkinny::NT,
                   TileSkinny::SMEM, s, pdl_gemm, args);
    else
        launch_pdl(f32p::f32_gemm_kernel<Tile8x4, false>, dim3((unsigned)ctas), Tile8x4::NT, Tile8x4::SMEM, s,
                   pdl_gemm, args);
    g_launches++;
    if (split) {   // the partial results summed into C in split order
        const int64_t rc = (d.M * d.N + 31) / 32;
        if (rc > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "output too large for one launch");
        launch_pdl(f32p::f32_split_reduce_kernel, dim3((unsigned)rc), 256, 0, s, true, ga,
                   (const float *)args.split_part, (int)d.ksplit);
        g_launches++;
    }
    RN_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

// The FP32 GEMM's tile for an M x N output (N <= M after the operand swap).
void f32p_tile(int64_t N, int *bm, int *bn) {
    *bm = f32p_skinny(N) ? f32p::TileSkinny::BM : f32p::BM;
    *bn = f32p_skinny(N) ? f32p::TileSkinny::BN : f32p::BN;
}

// The contraction split of a few-column problem for the FP32 GEMM (0 if it
// is not one): enough CTAs to reach every SM, at least two k-tiles each.
int64_t f32p_skinny_split(const GettDesc &d) {
    if (!f32p_skinny(d.N)) return 0;
    const int64_t nkt = (d.K + f32p::BK - 1) / f32p::BK, tiles = d.tiles_m * d.tiles_n;
    return std::max<int64_t>(1, std::min<int64_t>((num_sms() + tiles - 1) / tiles, nkt / 2));
}

// Whether the packed FP32 GEMM of a problem takes the stream-K schedule.
// Measured on B300 against one CTA per tile (8 x 4 outputs a thread in both,
// operands in L2): stream-K pays where the tiles leave the SMs unevenly
// loaded and a tile has enough k-tiles to split -- 2000 x 300 x 333 (160
// tiles, 11 k-tiles; 148 SMs take one whole tile each and the other 12 are
// split over a second CTA per SM): 49.4 against 65.7 us; 704 x 704 x 1024
// (121 tiles, 32 k-tiles): 94.2 against 98.4 us.  It loses where the
// imbalance is small or a tile has few k-tiles: 4096 x 256 x 256 (256 tiles
// of 8 k-tiles) 53.3 against 49.2 us, 1000 x 700 x 200 (176 tiles of 7)
// 47.2 against 43.0, and on large problems (1024 x 32768 x 1024: 4.91
// against 4.52 ms).  Never with a sequential (one CTA per tile) reduction;
// the autotuner times both schedules on more shapes than this selects.
bool f32p_stream_k_pays(const GettDesc &d, int reduce_mode) {
    if (reduce_mode == kReduceSequential || f32p_skinny(d.N) || d.ksplit > 1) return false;
    const int64_t tiles = d.tiles_m * d.tiles_n, sms = num_sms();
    const int64_t nkt = (d.K + f32p::BK - 1) / f32p::BK;
    if (tiles >= 3 * sms) return false;
    // the busiest SM's tiles over the average
    const double per = (double)tiles / (double)sms, imbalance = std::ceil(per) / per;
    return (nkt >= 8 && imbalance >= 1.5) || (nkt >= 32 && imbalance >= 1.15);
}

// Whether the autotuner times the stream-K schedule of a problem: any
// problem with fewer than three rounds of tiles over the CTA slots and at
// least 4 k-tiles a tile (the cases where balance can pay for the pieces).
bool f32p_stream_k_worth_timing(const GettDesc &d, int reduce_mode) {
    if (reduce_mode == kReduceSequential || f32p_skinny(d.N) || d.ksplit > 1) return false;
    const int64_t tiles = d.tiles_m * d.tiles_n, slots = 2 * (int64_t)num_sms();
    return tiles < 3 * slots && (d.K + f32p::BK - 1) / f32p::BK >= 4;
}

// Workspace bytes of a packed-kind problem: its packed operands (and the
// stream-K partial tiles and counters, or a split contraction's partial
// results, of the packed FP32 GEMM), for any operand addresses.
size_t tc_workspace_bytes(const GettDesc &d, int mode) {
    if (mode == kPackedModeF32) return f32_geom(d).total;
    TcGeom g = tc_geom(d, mode);
    return g.narr * g.arrA + g.narr_b * g.arrB;
}

// The same for the operand addresses bound in d: no packed panels when both
// operands are read in place.
size_t tc_workspace_bytes_bound(const GettDesc &d, int mode) {
    if (mode != kPackedModeF32) return tc_workspace_bytes(d, mode);
    const bool da = tma_direct_ok(d.flags & kFlagADense, d.a, d.M, d.K, d.a_plane);
    const bool db = tma_direct_ok(d.flags & kFlagBDense, d.b, d.N, d.K, d.b_plane);
    return f32_geom(d, da && db).total;
}

// Zero what must start at zero in a fresh workspace of a packed-kind problem
// (the stream-K tile counters, at its start; each launch leaves them at zero
// again).
void tc_workspace_clear(const GettDesc &d, int mode, void *ws, cudaStream_t s) {
    if (mode != kPackedModeF32 || !(d.flags & kFlagStreamK)) return;
    const F32Geom g = f32_geom(d);
    RN_CHECK_CUDA(cudaMemsetAsync(ws, 0, g.count_bytes, s));
}

// Enqueue pack + GEMM for one tensor-core problem.  `ga` locates the
// problem's descriptor (by value or in device memory); ws holds
// tc_workspace_bytes(d, mode) bytes, 256-byte aligned.  pack_a / pack_b = false
// reuse the packed operand already in ws (same operand as the previous call).
// before_gemm, when set, is called after the pack launches and before the
// GEMM launch (e.g. to record a timing event around the GEMM alone).  pdl =
// false: the first kernel starts only after everything before it in the
// stream has completed (it follows a kernel that built its offset tables).
void launch_tc_problem(int mode, const GettDesc &d, const GroupArgs &ga, void *ws, cudaStream_t s,
                       bool pack_a, bool pack_b, const std::function<void()> &before_gemm, bool pdl) {
    const int64_t ctas = d.tiles_m * d.tiles_n * (mode == kPackedModeF32 ? std::max(1, d.ksplit) : 1);
    if (ctas <= 0) return;
    if (ctas > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "problem too large for one launch");
    if (mode == kPackedModeF32) {
        launch_f32(ga, d, ws, ctas, s, pack_a, pack_b, before_gemm, pdl);
        return;
    }
    const TcGeom g = tc_geom(d, mode);
    if (ctas > 0x7fffffffLL || g.Kpad / g.bk > 0x7fffffffLL || g.Mpad > 0x7fffffffLL || g.Npad > 0x7fffffffLL)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "problem too large for one tensor-core launch");
    switch (mode) {
        case tc::kTF32: launch_mode<tc::kTF32>(ga, g, ws, ctas, s, pack_a, pack_b, before_gemm); break;
        case tc::kTF32x3: launch_mode<tc::kTF32x3>(ga, g, ws, ctas, s, pack_a, pack_b, before_gemm); break;
        default: launch_mode<tc::kBF16x3>(ga, g, ws, ctas, s, pack_a, pack_b, before_gemm); break;
    }
}

// A wait on an mbarrier that nothing completes, bounded by `budget` cycles:
// exercises the timeout path (status word set, kernel returns) without any
// fault.  Used by rosnet_selftest_timeout.
__global__ void selftest_wait_kernel(long long budget, int32_t *result) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = tc::mbar_try(&bar, 0);
        const long long t0 = clock64();
        while (!ok) {
            if (clock64() - t0 > budget) {
                atomicExch(&g_dev_status, kDevErrTimeout);
                break;
            }
            __nanosleep(64);
            ok = tc::mbar_try(&bar, 0);
        }
        *result = ok ? 1 : 0;
    }
}

// Read and clear the device status word (0 = no kernel gave up a wait).
int32_t take_device_status() {
    int32_t v = 0, z = 0;
    RN_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(v)));
    if (v) RN_CHECK_CUDA(cudaMemcpyToSymbol(g_dev_status, &z, sizeof(z)));
    return v;
}

}  // namespace rosnet

extern "C" rosnet_status rosnet_selftest_timeout(int64_t budget_cycles, void *stream) {
    using namespace rosnet;
    RN_API_BEGIN
    if (budget_cycles < 0 || budget_cycles > 4000000000LL)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "budget must be in [0, 4e9] cycles");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf r(sizeof(int32_t), s);
    selftest_wait_kernel<<<1, 32, 0, s>>>((long long)budget_cycles, (int32_t *)r.p);
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
    return ROSNET_OK;
    RN_API_END
}
