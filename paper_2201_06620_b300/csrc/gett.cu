// The pairwise blocked tensordot on CUDA cores.
//
// Sec. II-C computes each output block as the sum over the pairs of A and B
// blocks matched on the contracted-index block coordinates of the local
// contraction of each pair.  Here every logical axis of a block tensor
// contributes two index digits (its block coordinate and its position inside
// the block), each with its own element stride in the block-major layout.
// Classifying the digits of all axes as M (free in A), N (free in B) or K
// (contracted) turns the whole blocked contraction into one GEMM-shaped loop
// nest C[m, n] = sum_k A[m, k] B[k, n] whose operands are addressed through
// offset tables.  The K digits include the contracted block coordinates, so
// the K loop of one output tile walks the matched block pairs (steps 1-2)
// and the intra-block contraction (step 3), and keeps the partial sums of all
// pairs in registers (step 4); no transpose pass and no partial block ever
// reaches memory.  The order of the sum over pairs is free (Sec. IV-A).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>

#include "internal.h"
#include "gett_common.cuh"

namespace rosnet {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// planner: the GEMM view
// ---------------------------------------------------------------------------
namespace {

// Digits of one logical axis of extent s carried by two layouts with block
// extents b0, b1 (nested): outer to inner, each with its stride in both.
void axis_digits(std::vector<Mode> &out, int64_t s, int64_t b0, int64_t g0, int64_t l0, int64_t b1,
                 int64_t g1, int64_t l1) {
    int64_t lo = std::min(b0, b1), hi = std::max(b0, b1);
    if (lo < 1 || hi % lo) RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "block extents are not nested");
    auto st = [](int64_t u, int64_t b, int64_t g, int64_t l) { return u >= b ? g * (u / b) : l * u; };
    const int64_t ext[3] = {s / hi, hi / lo, lo};
    const int64_t unit[3] = {hi, lo, 1};
    for (int i = 0; i < 3; ++i)
        if (ext[i] != 1) out.push_back(Mode{ext[i], st(unit[i], b0, g0, l0), st(unit[i], b1, g1, l1)});
}

// Order digits outermost-first by the stride in tensor `which` (0 or 1),
// then fuse neighbours that are contiguous in both tensors.
void order_and_fuse(std::vector<Mode> &ms, int which, ModeList &out) {
    std::stable_sort(ms.begin(), ms.end(), [which](const Mode &x, const Mode &y) {
        int64_t a = which ? x.s1 : x.s0, b = which ? y.s1 : y.s0;
        return a > b;
    });
    out.n = 0;
    for (const Mode &q : ms) {
        if (out.n > 0) {
            Mode &p = out.m[out.n - 1];
            if (p.s0 == q.s0 * q.ext && p.s1 == q.s1 * q.ext) {
                p.ext *= q.ext;
                p.s0 = q.s0;
                p.s1 = q.s1;
                continue;
            }
        }
        if (out.n >= kMaxModes) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "too many index digits");
        out.m[out.n++] = q;
    }
}

int64_t min_stride(const std::vector<Mode> &ms, int which) {
    int64_t m = INT64_MAX;
    for (const Mode &x : ms) m = std::min(m, which ? x.s1 : x.s0);
    return m;
}

}  // namespace

GettView make_view(const Layout &A, const Layout &B, const Layout &C, int naxes, const int *axa,
                   const int *axb) {
    bool ca[kMaxRank] = {false}, cb[kMaxRank] = {false};
    for (int i = 0; i < naxes; ++i) {
        ca[axa[i]] = true;
        cb[axb[i]] = true;
    }
    std::vector<Mode> mM, mN, mK;
    int p = 0;  // axis of C
    for (int i = 0; i < A.rank; ++i) {
        if (ca[i]) continue;
        axis_digits(mM, A.shape[i], A.block[i], A.gstride[i], A.lstride[i], C.block[p],
                    C.gstride[p], C.lstride[p]);
        ++p;
    }
    for (int i = 0; i < B.rank; ++i) {
        if (cb[i]) continue;
        axis_digits(mN, B.shape[i], B.block[i], B.gstride[i], B.lstride[i], C.block[p],
                    C.gstride[p], C.lstride[p]);
        ++p;
    }
    for (int i = 0; i < naxes; ++i) {
        int x = axa[i], y = axb[i];
        axis_digits(mK, A.shape[x], A.block[x], A.gstride[x], A.lstride[x], B.block[y], B.gstride[y],
                    B.lstride[y]);
    }
    GettView v;
    // A's unit-stride digit decides whether A tiles are read along m or k;
    // likewise B along n or k.
    v.a_m_fast = !mM.empty() && min_stride(mM, 0) < min_stride(mK, 0);
    v.b_n_fast = !mN.empty() && min_stride(mN, 0) < min_stride(mK, 1);
    v.c_n_fast = mM.empty() || (!mN.empty() && min_stride(mN, 1) < min_stride(mM, 1));
    order_and_fuse(mM, 0, v.M);
    order_and_fuse(mN, 0, v.N);
    order_and_fuse(mK, v.a_m_fast ? 1 : 0, v.K);
    v.Mtot = v.M.total();
    v.Ntot = v.N.total();
    v.Ktot = v.K.total();
    return v;
}

size_t table_entries(const GettView &v) {
    return (size_t)(2 * v.Mtot + 2 * v.Ntot + 2 * v.Ktot);
}

// offsets of every index value of one class in its two tensors
__global__ void __launch_bounds__(256) build_table_kernel(ModeList ml, int64_t total,
                                                          int64_t *__restrict__ out0,
                                                          int64_t *__restrict__ out1) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i, o0 = 0, o1 = 0;
        for (int j = ml.n - 1; j >= 0; --j) {
            int64_t x = ml.m[j].ext;
            int64_t d;
            if ((x & (x - 1)) == 0) {
                d = r & (x - 1);
                r >>= __popcll(x - 1);
            } else {
                d = r % x;
                r /= x;
            }
            o0 += d * ml.m[j].s0;
            o1 += d * ml.m[j].s1;
        }
        out0[i] = o0;
        out1[i] = o1;
    }
}

static void launch_table(const ModeList &ml, int64_t total, int64_t *o0, int64_t *o1,
                         cudaStream_t s) {
    if (total <= 0) return;
    int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8);
    build_table_kernel<<<(int)blocks, 256, 0, s>>>(ml, total, o0, o1);
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

void launch_build_tables(const GettView &v, int64_t *t, cudaStream_t s) {
    launch_table(v.M, v.Mtot, t, t + v.Mtot, s);
    t += 2 * v.Mtot;
    launch_table(v.N, v.Ntot, t, t + v.Ntot, s);
    t += 2 * v.Ntot;
    launch_table(v.K, v.Ktot, t, t + v.Ktot, s);
}

void fill_desc_tables(GettDesc &d, const GettView &v, const int64_t *t) {
    fill_desc_tables(d, v, t, t + 2 * v.Mtot, t + 2 * v.Mtot + 2 * v.Ntot);
}

void host_mode_record(const ModeList &ml, int64_t *out) {
    out[0] = ml.n;
    for (int j = 0; j < ml.n; ++j) {
        out[1 + 3 * j] = ml.m[j].ext;
        out[2 + 3 * j] = ml.m[j].s0;
        out[3 + 3 * j] = ml.m[j].s1;
    }
}

__global__ void write_record_kernel(ModeList ml, int64_t *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[0] = ml.n;
        for (int j = 0; j < ml.n; ++j) {
            out[1 + 3 * j] = ml.m[j].ext;
            out[2 + 3 * j] = ml.m[j].s0;
            out[3 + 3 * j] = ml.m[j].s1;
        }
    }
}

TableLayout table_layout(const GettView &v, int record_class) {
    TableLayout L;
    L.record_class = record_class;
    const ModeList *ml[3] = {&v.M, &v.N, &v.K};
    const int64_t tot[3] = {v.Mtot, v.Ntot, v.Ktot};
    int64_t o = 0;
    for (int c = 0; c < 3; ++c) {
        L.off[c] = o;
        o += c == record_class ? record_entries(*ml[c]) : 2 * tot[c];
    }
    L.entries = o;
    return L;
}

void launch_build_tables(const GettView &v, const TableLayout &L, int64_t *t, cudaStream_t s) {
    const ModeList *ml[3] = {&v.M, &v.N, &v.K};
    const int64_t tot[3] = {v.Mtot, v.Ntot, v.Ktot};
    for (int c = 0; c < 3; ++c) {
        if (c == L.record_class) {
            write_record_kernel<<<1, 32, 0, s>>>(*ml[c], t + L.off[c]);
            g_launches++;
            RN_CHECK_CUDA(cudaGetLastError());
        } else {
            launch_table(*ml[c], tot[c], t + L.off[c], t + L.off[c] + tot[c], s);
        }
    }
}

void fill_desc_tables(GettDesc &d, const GettView &v, const int64_t *tm, const int64_t *tn,
                      const int64_t *tk) {
    d.offAM = tm;
    d.offCM = tm + v.Mtot;
    d.offBN = tn;
    d.offCN = tn + v.Ntot;
    d.offAK = tk;
    d.offBK = tk + v.Ktot;
    d.M = v.Mtot;
    d.N = v.Ntot;
    d.K = v.Ktot;
    // digits whose strides in one tensor form a row-major sequence starting at
    // `base` (the table of that class is then i -> i * base)
    auto row_major = [](const ModeList &ml, int which, int64_t base) {
        int64_t e = base;
        for (int i = ml.n - 1; i >= 0; --i) {
            if ((which ? ml.m[i].s1 : ml.m[i].s0) != e) return false;
            e *= ml.m[i].ext;
        }
        return true;
    };
    const bool a_dense = row_major(v.M, 0, 1) && row_major(v.K, 0, v.Mtot);
    const bool b_dense = row_major(v.N, 0, 1) && row_major(v.K, 1, v.Ntot);
    // vector access (gett_gate_kernel): the innermost mode of a class is a
    // unit-stride run whose extent is a multiple of 8, and every other offset
    // of the tensor involved is a multiple of 4 elements (16 bytes)
    auto mult4 = [](const ModeList &ml, int which, int skip_inner) {
        for (int i = 0; i < ml.n - skip_inner; ++i)
            if ((which ? ml.m[i].s1 : ml.m[i].s0) % 4) return false;
        return true;
    };
    auto run8 = [&](const ModeList &ml, int which, int64_t stride) {
        return ml.n > 0 && (which ? ml.m[ml.n - 1].s1 : ml.m[ml.n - 1].s0) == stride &&
               ml.m[ml.n - 1].ext % 8 == 0 && mult4(ml, which, 1);
    };
    // C with class `in` innermost and dense (offsets 0 .. tot - 1), the
    // innermost mode of class `out` right above it in runs of 8
    auto inner = [&](const ModeList &in, int64_t tot, const ModeList &out) {
        const bool dense = in.n == 0 || (in.n == 1 && in.m[0].s1 == 1);
        return dense && (tot == 1 || tot == 2 || tot == 4) && run8(out, 1, tot);
    };
    int vec = 0;
    if (run8(v.M, 0, 1) && mult4(v.K, 0, 0)) vec |= kFlagAMVec;
    if (run8(v.N, 0, 1) && mult4(v.K, 1, 0)) vec |= kFlagBNVec;
    if (run8(v.M, 1, 1) && mult4(v.N, 1, 0)) vec |= kFlagCMVec;
    if (run8(v.N, 1, 1) && mult4(v.M, 1, 0)) vec |= kFlagCNVec;
    if (inner(v.N, v.Ntot, v.M)) vec |= kFlagCNInner;
    if (inner(v.M, v.Mtot, v.N)) vec |= kFlagCMInner;
    d.flags = (v.a_m_fast ? kFlagAMFast : 0) | (v.b_n_fast ? kFlagBNFast : 0) |
              (v.c_n_fast ? kFlagCNFast : 0) | (a_dense ? kFlagADense : 0) | (b_dense ? kFlagBDense : 0) | vec;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cmac(T &cr, T &ci, T ar, T ai, T br, T bi) {
    cr = fma(ar, br, cr);
    cr = fma(-ai, bi, cr);
    ci = fma(ar, bi, ci);
    ci = fma(ai, br, ci);
}

// (m, n) of output o of a thread-per-output kernel: n fastest when B or C
// are contiguous along n, else m fastest.
__device__ __forceinline__ void out_coords(const GettDesc &d, int64_t o, int64_t &m, int64_t &n) {
    if (d.flags & (kFlagBNFast | kFlagCNFast)) {
        n = o % d.N;
        m = o / d.N;
    } else {
        m = o % d.M;
        n = o / d.M;
    }
}

// One thread per output entry; the (short) K loop runs in registers.
template <typename T>
__global__ void __launch_bounds__(256) gett_small_kernel(const __grid_constant__ GroupArgs g) {
    __shared__ GettDesc sd;
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x - sd.tile_begin;
    const int64_t o = tile * 256 + threadIdx.x;
    const int64_t M = sd.M, N = sd.N, K = sd.K;
    const bool live = o < M * N;
    int64_t m = 0, n = 0, am = 0, bn = 0, ic = 0;
    if (live) {
        out_coords(sd, o, m, n);
        am = sd.offAM[m];
        bn = sd.offBN[n];
        ic = sd.offCM[m] + sd.offCN[n];
    }
    grid_dep_wait();
    if (!live) return;
    const T *__restrict__ A = (const T *)sd.a;
    const T *__restrict__ B = (const T *)sd.b;
    const int64_t *__restrict__ offAK = sd.offAK;
    const int64_t *__restrict__ offBK = sd.offBK;
    const int64_t ap = sd.a_plane, bp = sd.b_plane;
    T sr = 0, si = 0;
#pragma unroll 4
    for (int64_t k = 0; k < K; ++k) {
        const int64_t ia = am + offAK[k], ib = bn + offBK[k];
        cmac(sr, si, A[ia], A[ia + ap], B[ib], B[ib + bp]);
    }
    T *C = (T *)sd.c;
    C[ic] = sr;
    C[ic + sd.c_plane] = si;
}

// The leaf-side small steps of a plan in one launch.  CTA c runs one
// connected group of them -- steps whose operands are leaves or earlier steps
// of the same group, a subtree of the contraction -- level by level: the
// steps of a level are independent of one another, their output entries are
// spread over all the CTA's threads (one thread per entry, the K loop in
// registers, as gett_small_kernel), and a barrier separates levels, so every
// step reads only outputs its own CTA wrote before the barrier (operands are
// read with coherent loads, not the read-only path).  No CTA waits for
// another.  The group's descriptors are staged in shared memory once.
// prog: [G, then G + 1 level offsets (CTA c owns levels [prog[1 + c],
// prog[2 + c])), then per level (first descriptor, descriptor count)]; a
// CTA's descriptors are contiguous, at most kForestMaxSteps of them.
struct ForestDesc {
    const void *a, *b;
    void *c;
    int64_t a_plane, b_plane, c_plane;
    const int64_t *offAM, *offBN, *offAK, *offBK, *offCM, *offCN;
    int64_t M, N, K;
    int64_t pre;     // output entries of the level's earlier steps
    int64_t flags;
};

template <typename T>
__global__ void __launch_bounds__(kForestThreads) gett_forest_kernel(const GettDesc *descs, const int64_t *prog) {
    __shared__ ForestDesc fd[kForestMaxSteps];
    grid_dep_launch();
    grid_dep_wait();   // leaves and descriptors may come from earlier work on the stream
    const int64_t G = prog[0];
    const int64_t *lv = prog + G + 2;
    const int64_t l0 = prog[1 + blockIdx.x], l1 = prog[2 + blockIdx.x];
    const int64_t d0 = lv[2 * l0], nd = lv[2 * (l1 - 1)] + lv[2 * (l1 - 1) + 1] - d0;
    for (int64_t j = threadIdx.x; j < nd; j += kForestThreads) {
        const GettDesc &d = descs[d0 + j];
        ForestDesc &f = fd[j];
        f.a = d.a; f.b = d.b; f.c = d.c;
        f.a_plane = d.a_plane; f.b_plane = d.b_plane; f.c_plane = d.c_plane;
        f.offAM = d.offAM; f.offBN = d.offBN; f.offAK = d.offAK; f.offBK = d.offBK;
        f.offCM = d.offCM; f.offCN = d.offCN;
        f.M = d.M; f.N = d.N; f.K = d.K;
        f.flags = d.flags;
    }
    __syncthreads();
    if (threadIdx.x == 0)   // per level, the running count of output entries
        for (int64_t l = l0; l < l1; ++l) {
            int64_t run = 0;
            for (int64_t j = lv[2 * l] - d0; j < lv[2 * l] - d0 + lv[2 * l + 1]; ++j) {
                fd[j].pre = run;
                run += fd[j].M * fd[j].N;
            }
        }
    __syncthreads();
    for (int64_t l = l0; l < l1; ++l) {
        const int jb = (int)(lv[2 * l] - d0), je = jb + (int)lv[2 * l + 1];
        const int64_t total = fd[je - 1].pre + fd[je - 1].M * fd[je - 1].N;
        for (int64_t i = threadIdx.x; i < total; i += kForestThreads) {
            int lo = jb, hi = je - 1;   // the last step whose entries start at or before i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (fd[mid].pre <= i) lo = mid;
                else hi = mid - 1;
            }
            const ForestDesc &f = fd[lo];
            const int64_t o = i - f.pre;
            int64_t m, n;
            if (f.flags & (kFlagBNFast | kFlagCNFast)) {
                n = o % f.N;
                m = o / f.N;
            } else {
                m = o % f.M;
                n = o / f.M;
            }
            const T *A = (const T *)f.a;
            const T *B = (const T *)f.b;
            const int64_t am = __ldg(f.offAM + m), bn = __ldg(f.offBN + n);
            T sr = 0, si = 0;
#pragma unroll 4
            for (int64_t k = 0; k < f.K; ++k) {
                const int64_t ia = am + __ldg(f.offAK + k), ib = bn + __ldg(f.offBK + k);
                cmac(sr, si, A[ia], A[ia + f.a_plane], B[ib], B[ib + f.b_plane]);
            }
            T *C = (T *)f.c;
            const int64_t ic = __ldg(f.offCM + m) + __ldg(f.offCN + n);
            C[ic] = sr;
            C[ic + f.c_plane] = si;
        }
        __syncthreads();   // this level's outputs are visible to the next level
    }
}

// One warp per output entry; lanes split the K loop, shuffle reduction.
template <typename T>
__global__ void __launch_bounds__(256) gett_warpk_kernel(const __grid_constant__ GroupArgs g) {
    __shared__ GettDesc sd;
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x - sd.tile_begin;
    const int64_t o = tile * 8 + (threadIdx.x >> 5);
    const int64_t M = sd.M, N = sd.N, K = sd.K;
    const bool live = o < M * N;
    int64_t m = 0, n = 0, am = 0, bn = 0;
    if (live) {
        out_coords(sd, o, m, n);
        am = sd.offAM[m];
        bn = sd.offBN[n];
    }
    grid_dep_wait();
    if (!live) return;
    const T *__restrict__ A = (const T *)sd.a;
    const T *__restrict__ B = (const T *)sd.b;
    const int64_t ap = sd.a_plane, bp = sd.b_plane;
    T sr = 0, si = 0;
    for (int64_t k = lane; k < K; k += 32) {
        const int64_t ia = am + sd.offAK[k], ib = bn + sd.offBK[k];
        cmac(sr, si, A[ia], A[ia + ap], B[ib], B[ib + bp]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) {
        T *C = (T *)sd.c;
        const int64_t ic = sd.offCM[m] + sd.offCN[n];
        C[ic] = sr;
        C[ic + sd.c_plane] = si;
    }
}

// One cluster of kDotCTAs CTAs per output entry for very long contractions
// with few outputs (e.g. the final scalar of a network: an amplitude): the
// cluster's threads stride over K with four independent loads in flight
// each, every CTA reduces its threads' sums in a fixed order, and CTA 0 of
// the cluster adds the CTAs' sums in rank order through distributed shared
// memory.  Products and sums are taken in FP64 whatever the operands' type
// (a product of two floats is exact in double), so the final reduction of an
// amplitude adds no FP32 rounding; the result is rounded once to C's type.
// One launch, no workspace, deterministic.
template <typename T>
__global__ void __cluster_dims__(kDotCTAs, 1, 1) __launch_bounds__(256)
    gett_dot_kernel(const __grid_constant__ GroupArgs g) {
    __shared__ GettDesc sd;
    __shared__ double red[2][8];
    __shared__ double cta_sum[2];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    // tile_begin of every problem is a multiple of kDotCTAs, so one cluster
    // never spans two problems
    const int64_t o = ((int64_t)blockIdx.x - sd.tile_begin) / kDotCTAs;
    int64_t m, n;
    out_coords(sd, o, m, n);
    const T *__restrict__ A = (const T *)sd.a;
    const T *__restrict__ B = (const T *)sd.b;
    const int64_t *__restrict__ offAK = sd.offAK;
    const int64_t *__restrict__ offBK = sd.offBK;
    const int64_t am = sd.offAM[m], bn = sd.offBN[n], K = sd.K;
    const int64_t ap = sd.a_plane, bp = sd.b_plane;
    constexpr int64_t stride = 256 * kDotCTAs;
    grid_dep_wait();
    double sr = 0, si = 0;
    auto mac = [&](T ar, T ai, T br, T bi) {
        cmac<double>(sr, si, (double)ar, (double)ai, (double)br, (double)bi);
    };
    int64_t k = (int64_t)rank * 256 + threadIdx.x;
    for (; k + 3 * stride < K; k += 4 * stride) {
        int64_t ia[4], ib[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ia[u] = am + __ldg(offAK + k + stride * u);
            ib[u] = bn + __ldg(offBK + k + stride * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) mac(__ldg(A + ia[u]), __ldg(A + ia[u] + ap), __ldg(B + ib[u]), __ldg(B + ib[u] + bp));
    }
    for (; k < K; k += stride) {
        const int64_t ia = am + offAK[k], ib = bn + offBK[k];
        mac(A[ia], A[ia + ap], B[ib], B[ib + bp]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = sr;
        red[1][w] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0, ti = 0;
        for (int j = 0; j < 8; ++j) {
            tr += red[0][j];
            ti += red[1][j];
        }
        cta_sum[0] = tr;
        cta_sum[1] = ti;
    }
    cluster.sync();   // every CTA's sum is visible to the cluster
    if (rank == 0 && threadIdx.x == 0) {
        double tr = 0, ti = 0;
        for (int r = 0; r < kDotCTAs; ++r) {
            const double *p = cluster.map_shared_rank(cta_sum, r);
            tr += p[0];
            ti += p[1];
        }
        T *C = (T *)sd.c;
        const int64_t ic = sd.offCM[m] + sd.offCN[n];
        C[ic] = (T)tr;
        C[ic + sd.c_plane] = (T)ti;
    }
    cluster.sync();   // no CTA leaves while CTA 0 may still read its sum
}

// Low arithmetic intensity: C[m, n] = sum_k A[m, k] B[k, n] for K, N <= 4
// and M large -- a one- or two-qubit gate applied along some axes of a big
// tensor, a projection, a vector-like block.  The work is streaming A and C
// through HBM once.  Each thread takes V consecutive m (a unit-stride run in
// A and in C, kFlagAMVec and kFlagCMVec / kFlagCNInner) and reads them with
// 16-byte loads, two planes per contracted index; the whole small operand B
// sits in registers; C leaves with 16-byte stores: V values per n along C's
// m run, or the V x N block when C's n index is innermost.  The offsets of
// the M index come from its mode record (a few shifts per thread, no table
// as large as the tensor); the other tables hold at most 4 entries.  Planes
// that do not start on 16-byte boundaries are read and written element by
// element instead.
// Whether a gate kind's CTAs loop over runs of rows (the kinds with a side
// of 4, whose 90-128 registers fit at most two CTAs per SM) rather than take
// one run per thread.
constexpr bool gate_loops(int nk, int nn) { return nk == 4 || nn == 4; }

template <int NK, int NN>
__global__ void __launch_bounds__(256) gett_gate_kernel(const __grid_constant__ GroupArgs g) {
    if constexpr (!gate_loops(NK, NN)) {   // one run of rows per thread
    constexpr int V = NK * NN >= 8 ? 4 : 8;   // rows per thread
    constexpr int NV = V / 4;                 // float4 per plane per row run
    __shared__ GettDesc sd;
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    const int64_t m0 = (((int64_t)blockIdx.x - sd.tile_begin) * 256 + threadIdx.x) * V;
    const bool live = m0 < sd.M;
    // offsets of row m0 in A and C from the mode record of the M class
    int64_t am = 0, cm = 0, ak[NK], cn[NN];
    if (live) {
        const int64_t *rec = sd.offAM;
        int64_t r = m0;
        for (int j = (int)__ldg(rec) - 1; j >= 0; --j) {
            const int64_t ext = __ldg(rec + 1 + 3 * j);
            int64_t dg;
            if ((ext & (ext - 1)) == 0) {
                dg = r & (ext - 1);
                r >>= __popcll(ext - 1);
            } else {
                dg = r % ext;
                r /= ext;
            }
            am += dg * __ldg(rec + 2 + 3 * j);
            cm += dg * __ldg(rec + 3 + 3 * j);
        }
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) ak[k] = __ldg(sd.offAK + k);
#pragma unroll
    for (int n = 0; n < NN; ++n) cn[n] = __ldg(sd.offCN + n);
    grid_dep_wait();   // A and B may be the previous kernel's results
    if (!live) return;
    const float *__restrict__ A = (const float *)sd.a;
    const float *__restrict__ B = (const float *)sd.b;
    float gr[NK][NN], gi[NK][NN];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            const int64_t o = __ldg(sd.offBK + k) + __ldg(sd.offBN + n);
            gr[k][n] = B[o];
            gi[k][n] = B[o + sd.b_plane];
        }
    float *C = (float *)sd.c;
    const int64_t cp = sd.c_plane;
    // every offset is a multiple of 4 elements (the vector flags); 16-byte
    // accesses need the planes to start on 16-byte boundaries too
    const bool vec = (((uintptr_t)A | (uintptr_t)C) & 15) == 0 && ((sd.a_plane | cp) & 3) == 0;
    float xr[NK][V], xi[NK][V];
    if (vec) {
#pragma unroll
        for (int k = 0; k < NK; ++k)
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const float4 r = __ldcs(reinterpret_cast<const float4 *>(A + am + ak[k]) + q);
                const float4 i = __ldcs(reinterpret_cast<const float4 *>(A + am + ak[k] + sd.a_plane) + q);
                xr[k][4 * q] = r.x; xr[k][4 * q + 1] = r.y; xr[k][4 * q + 2] = r.z; xr[k][4 * q + 3] = r.w;
                xi[k][4 * q] = i.x; xi[k][4 * q + 1] = i.y; xi[k][4 * q + 2] = i.z; xi[k][4 * q + 3] = i.w;
            }
    } else {
#pragma unroll
        for (int k = 0; k < NK; ++k)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                xr[k][v] = A[am + ak[k] + v];
                xi[k][v] = A[am + ak[k] + v + sd.a_plane];
            }
    }
    float cr[NN][V], ci[NN][V];
#pragma unroll
    for (int n = 0; n < NN; ++n)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int k = 0; k < NK; ++k) cmac(sr, si, xr[k][v], xi[k][v], gr[k][n], gi[k][n]);
            cr[n][v] = sr;
            ci[n][v] = si;
        }
    if (sd.flags & kFlagCMVec) {   // each n: V consecutive outputs along m
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            float *o = C + cm + cn[n];
            if (vec) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    __stcs(reinterpret_cast<float4 *>(o) + q,
                           make_float4(cr[n][4 * q], cr[n][4 * q + 1], cr[n][4 * q + 2], cr[n][4 * q + 3]));
                    __stcs(reinterpret_cast<float4 *>(o + cp) + q,
                           make_float4(ci[n][4 * q], ci[n][4 * q + 1], ci[n][4 * q + 2], ci[n][4 * q + 3]));
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    o[v] = cr[n][v];
                    o[v + cp] = ci[n][v];
                }
            }
        }
    } else {                       // n innermost: the V x NN block is contiguous
        constexpr int E = V * NN;
        float er[E], ei[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            er[e] = cr[e % NN][e / NN];
            ei[e] = ci[e % NN][e / NN];
        }
        if (vec) {
#pragma unroll
            for (int q = 0; q < E / 4; ++q) {
                __stcs(reinterpret_cast<float4 *>(C + cm) + q,
                       make_float4(er[4 * q], er[4 * q + 1], er[4 * q + 2], er[4 * q + 3]));
                __stcs(reinterpret_cast<float4 *>(C + cm + cp) + q,
                       make_float4(ei[4 * q], ei[4 * q + 1], ei[4 * q + 2], ei[4 * q + 3]));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                C[cm + e] = er[e];
                C[cm + e + cp] = ei[e];
            }
        }
    }
    } else {   // the problem's resident CTAs loop over the runs
    constexpr int V = NK * NN >= 8 ? 4 : 8;   // rows per thread
    constexpr int NV = V / 4;                 // float4 per plane per row run
    constexpr int kRecMax = 1 + 3 * 128;      // a mode record of up to 128 modes in shared memory
    __shared__ GettDesc sd;
    __shared__ int64_t rec[kRecMax];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    // the M class's mode record into shared memory (read by every run; a
    // longer one is read from global memory)
    const int64_t nrec = 1 + 3 * __ldg(sd.offAM);
    const int64_t *rp = nrec <= kRecMax ? rec : sd.offAM;
    if (nrec <= kRecMax)
        for (int e = threadIdx.x; e < nrec; e += 256) rec[e] = __ldg(sd.offAM + e);
    int64_t ak[NK], cn[NN], bo[NK][NN];
#pragma unroll
    for (int k = 0; k < NK; ++k) ak[k] = __ldg(sd.offAK + k);
#pragma unroll
    for (int n = 0; n < NN; ++n) cn[n] = __ldg(sd.offCN + n);
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int n = 0; n < NN; ++n) bo[k][n] = __ldg(sd.offBK + k) + __ldg(sd.offBN + n);
    __syncthreads();
    grid_dep_wait();   // A and B may be the previous kernel's results
    const float *__restrict__ A = (const float *)sd.a;
    const float *__restrict__ B = (const float *)sd.b;
    float gr[NK][NN], gi[NK][NN];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int n = 0; n < NN; ++n) {
            gr[k][n] = B[bo[k][n]];
            gi[k][n] = B[bo[k][n] + sd.b_plane];
        }
    float *C = (float *)sd.c;
    const int64_t cp = sd.c_plane;
    // every offset is a multiple of 4 elements (the vector flags); 16-byte
    // accesses need the planes to start on 16-byte boundaries too
    const bool vec = (((uintptr_t)A | (uintptr_t)C) & 15) == 0 && ((sd.a_plane | cp) & 3) == 0;
    // the problem's CTAs stay resident (as many as fit at once) and each
    // thread takes runs t, t + stride, ... of V rows: the descriptor, the
    // record and the gate are read once, and the loads of the next run
    // follow the stores of the last without a CTA's prologue between them
    const int64_t stride = sd.tiles_m * 256;
    for (int64_t t = ((int64_t)blockIdx.x - sd.tile_begin) * 256 + threadIdx.x; t * V < sd.M; t += stride) {
        const int64_t m0 = t * V;
        // offsets of row m0 in A and C from the mode record of the M class
        int64_t am = 0, cm = 0, r = m0;
        for (int jm = (int)rp[0] - 1; jm >= 0; --jm) {
            const int64_t ext = rp[1 + 3 * jm];
            int64_t dg;
            if ((ext & (ext - 1)) == 0) {
                dg = r & (ext - 1);
                r >>= __popcll(ext - 1);
            } else {
                dg = r % ext;
                r /= ext;
            }
            am += dg * rp[2 + 3 * jm];
            cm += dg * rp[3 + 3 * jm];
        }
        float xr[NK][V], xi[NK][V];
        if (vec) {
#pragma unroll
            for (int k = 0; k < NK; ++k)
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const float4 rr = __ldcs(reinterpret_cast<const float4 *>(A + am + ak[k]) + q);
                    const float4 ii = __ldcs(reinterpret_cast<const float4 *>(A + am + ak[k] + sd.a_plane) + q);
                    xr[k][4 * q] = rr.x; xr[k][4 * q + 1] = rr.y; xr[k][4 * q + 2] = rr.z; xr[k][4 * q + 3] = rr.w;
                    xi[k][4 * q] = ii.x; xi[k][4 * q + 1] = ii.y; xi[k][4 * q + 2] = ii.z; xi[k][4 * q + 3] = ii.w;
                }
        } else {
#pragma unroll
            for (int k = 0; k < NK; ++k)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    xr[k][v] = A[am + ak[k] + v];
                    xi[k][v] = A[am + ak[k] + v + sd.a_plane];
                }
        }
        float cr[NN][V], ci[NN][V];
#pragma unroll
        for (int n = 0; n < NN; ++n)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int k = 0; k < NK; ++k) cmac(sr, si, xr[k][v], xi[k][v], gr[k][n], gi[k][n]);
                cr[n][v] = sr;
                ci[n][v] = si;
            }
        if (sd.flags & kFlagCMVec) {   // each n: V consecutive outputs along m
#pragma unroll
            for (int n = 0; n < NN; ++n) {
                float *o = C + cm + cn[n];
                if (vec) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        __stcs(reinterpret_cast<float4 *>(o) + q,
                               make_float4(cr[n][4 * q], cr[n][4 * q + 1], cr[n][4 * q + 2], cr[n][4 * q + 3]));
                        __stcs(reinterpret_cast<float4 *>(o + cp) + q,
                               make_float4(ci[n][4 * q], ci[n][4 * q + 1], ci[n][4 * q + 2], ci[n][4 * q + 3]));
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        o[v] = cr[n][v];
                        o[v + cp] = ci[n][v];
                    }
                }
            }
        } else {                       // n innermost: the V x NN block is contiguous
            constexpr int E = V * NN;
            float er[E], ei[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                er[e] = cr[e % NN][e / NN];
                ei[e] = ci[e % NN][e / NN];
            }
            if (vec) {
#pragma unroll
                for (int q = 0; q < E / 4; ++q) {
                    __stcs(reinterpret_cast<float4 *>(C + cm) + q,
                           make_float4(er[4 * q], er[4 * q + 1], er[4 * q + 2], er[4 * q + 3]));
                    __stcs(reinterpret_cast<float4 *>(C + cm + cp) + q,
                           make_float4(ei[4 * q], ei[4 * q + 1], ei[4 * q + 2], ei[4 * q + 3]));
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    C[cm + e] = er[e];
                    C[cm + e + cp] = ei[e];
                }
            }
        }
    }
    }
}

// Sum of the split-K partials into C, in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) gett_reduce_kernel(const __grid_constant__ GroupArgs g) {
    // 32 outputs per CTA; warp w sums partials w, w + 8, w + 16, ... of its
    // lane's output (coalesced across lanes, independent loads in flight),
    // then warp 0 adds the eight sums in warp order: a fixed order, so the
    // result does not depend on scheduling.
    __shared__ GettDesc sd;
    __shared__ T red[2][8][33];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    grid_dep_wait();
    const int64_t MN = sd.M * sd.N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t o = ((int64_t)blockIdx.x - sd.tile_begin) * 32 + lane;
    const T *__restrict__ P = (const T *)sd.part;
    T sr = 0, si = 0;
    if (o < MN) {
#pragma unroll 4
        for (int s = w; s < sd.ksplit; s += 8) {
            sr += __ldg(P + (2 * (int64_t)s) * MN + o);
            si += __ldg(P + (2 * (int64_t)s + 1) * MN + o);
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
    const int64_t m = o / sd.N, n = o % sd.N;
    T *C = (T *)sd.c;
    const int64_t ic = sd.offCM[m] + sd.offCN[n];
    C[ic] = sr;
    C[ic + sd.c_plane] = si;
}

// C = 0 for the problems of a commutative split-K launch (4 entries per thread).
template <typename T>
__global__ void __launch_bounds__(256) gett_zero_kernel(const __grid_constant__ GroupArgs g) {
    __shared__ GettDesc sd;
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    grid_dep_wait();
    const int64_t MN = sd.M * sd.N;
    const int64_t o0 = ((int64_t)blockIdx.x - sd.tile_begin) * 1024 + threadIdx.x;
    T *C = (T *)sd.c;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t o = o0 + i * 256;
        if (o < MN) {
            const int64_t m = o / sd.N, n = o % sd.N;
            const int64_t ic = sd.offCM[m] + sd.offCN[n];
            C[ic] = 0;
            C[ic + sd.c_plane] = 0;
        }
    }
}

__device__ __forceinline__ void cp_async_el(void *smem, const void *gsrc, int bytes, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? bytes : 0;   // 0 source bytes: the shared word is zero-filled
    if (bytes == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// BM x BN output tile per CTA, 256 threads (BM / TM rows x BN / 4 columns of
// threads) each owning TM x 4 complex outputs.  A and B tiles of BK contracted indices are gathered
// element by element through the offset tables (consecutive threads take
// consecutive values of A's / B's unit-stride digit, so the gathers
// coalesce) with cp.async into a STAGES-deep shared-memory ring of planar
// re/im rows.  The K loop runs over every matched block pair and every
// intra-block index and keeps all partial sums in registers.  With split-K
// the CTA covers one contracted range and writes its partial tile to the
// workspace instead of C (summed by gett_reduce_kernel).
#ifndef ROSNET_TILED_KU
#define ROSNET_TILED_KU 2    // unroll of the two-row inner loop
#endif
#ifndef ROSNET_TILED_MINB
#define ROSNET_TILED_MINB 2  // resident CTAs per SM asked of the 64 x 64 FP32 tile
#endif

template <typename T, int BM, int BN, int BK, int STAGES>
struct TiledCfg {
    static constexpr int NT = 256;
    // threads: TXN along n (4 complex columns each), NT / TXN along m
    static constexpr int TN = 4, TXN = BN / TN, TY = NT / TXN, TM = BM / TY;
    static_assert(TXN * TY == NT && TM * TY == BM && TM % 4 == 0, "tile shape");
    static constexpr int LA = BM * BK / NT, LB = BN * BK / NT;
    static constexpr int PAD = 16 / sizeof(T);
    static constexpr int RA = BM + PAD, RB = BN + PAD;    // shared row lengths
    static constexpr int VA = TM * (int)sizeof(T) / 16;    // 16-byte vectors per row fragment
    static constexpr int VB = TN * (int)sizeof(T) / 16;
    static constexpr size_t smem = sizeof(T) * (size_t)STAGES * 2 * BK * (RA + RB);
    // one plane of the output tile is staged in the ring after the K loop
    static_assert((size_t)(BM + 1) * (BN + 1) * sizeof(T) <= smem, "epilogue staging exceeds the ring");
};

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};

// Epilogue of a register-tiled output tile (TM x TN complex values per thread
// at rows ty*TM.., columns tx*TN..): one plane at a time the tile goes through
// shared memory (cs: at least (BM + 1) * (BN + 1) elements, free for reuse)
// and out with the lanes of a warp along the destination's unit-stride
// dimension (n for split-K partials [m][n], else C's own), so stores coalesce
// whatever the output layout.  sCM / sCN: C offsets of the tile's rows and
// columns (unused for partials).  All 256 threads call it.
template <typename T, int BM, int BN, int TM, int TN>
__device__ __forceinline__ void store_tile(const GettDesc &sd, const T (&cr)[TM][TN], const T (&ci)[TM][TN], T *cs,
                                           const int64_t *sCM, const int64_t *sCN, int64_t m0, int64_t n0,
                                           int split, int ty, int tx) {
    constexpr int NT = 256;
    const int64_t M = sd.M, N = sd.N;
    const bool part = sd.part != nullptr;
    const bool m_fast = !part && !(sd.flags & kFlagCNFast);
    const bool atomic = sd.flags & kFlagAtomic;   // commutative split: order-free adds
    const int64_t MN = M * N;
    T *__restrict__ dst = part ? (T *)sd.part + (2 * (int64_t)split) * MN : (T *)sd.c;
    const int64_t dplane = part ? MN : sd.c_plane;
    const int ld = m_fast ? BM + 1 : BN + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll 1
    for (int pl = 0; pl < 2; ++pl) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int ml = ty * TM + i, nl = tx * TN + j;
                cs[m_fast ? nl * ld + ml : ml * ld + nl] = pl ? ci[i][j] : cr[i][j];
            }
        __syncthreads();
        T *__restrict__ out = dst + pl * dplane;
        if (m_fast) {   // lanes along m: this lane's rows' offsets once
            constexpr int UM = (BM + 31) / 32;
            int64_t cm[UM];
#pragma unroll
            for (int u = 0; u < UM; ++u) {
                const int ml = lane + 32 * u;
                cm[u] = (ml < BM && m0 + ml < M) ? sCM[ml] : -1;
            }
            for (int nl = warp; nl < BN; nl += NT / 32) {
                if (n0 + nl >= N) break;
                const int64_t cn = sCN[nl];
                const T *row = cs + nl * ld + lane;
#pragma unroll
                for (int u = 0; u < UM; ++u)
                    if (cm[u] >= 0) {
                        if (atomic) atomicAdd(out + cm[u] + cn, row[32 * u]);
                        else out[cm[u] + cn] = row[32 * u];
                    }
            }
        } else {        // lanes along n: this lane's columns' offsets once
            constexpr int UN = (BN + 31) / 32;
            int64_t cn[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int nl = lane + 32 * u;
                cn[u] = (nl < BN && n0 + nl < N) ? (part ? n0 + nl : sCN[nl]) : -1;
            }
            for (int ml = warp; ml < BM; ml += NT / 32) {
                const int64_t m = m0 + ml;
                if (m >= M) break;
                const int64_t base = part ? m * N : sCM[ml];
                const T *row = cs + ml * ld + lane;
#pragma unroll
                for (int u = 0; u < UN; ++u)
                    if (cn[u] >= 0) {
                        if (atomic) atomicAdd(out + base + cn[u], row[32 * u]);
                        else out[base + cn[u]] = row[32 * u];
                    }
            }
        }
        __syncthreads();   // the next plane reuses the staging area
    }
}

// The tile body, specialised on whether A (B) is read along m (n) or along k:
// with those known at compile time every thread's gather addresses reduce to
// one base offset per operand plus compile-time strides.
template <typename T, int BM, int BN, int BK, int STAGES, bool amf, bool bnf>
__device__ __forceinline__ void tiled_body(const GettDesc &sd, T *As, T *Bs, int64_t *sCM, int64_t *sCN) {
    using Cfg = TiledCfg<T, BM, BN, BK, STAGES>;
    using V = typename Vec16<T>::type;
    constexpr int NT = Cfg::NT, TM = Cfg::TM, TN = Cfg::TN, LA = Cfg::LA, LB = Cfg::LB;
    constexpr int RA = Cfg::RA, RB = Cfg::RB;
    constexpr int PA = BK * RA, PB = BK * RB;   // one plane of one stage
    const int tid = threadIdx.x;
    const int64_t tile = (int64_t)blockIdx.x - sd.tile_begin;
    const int64_t ntile = sd.tiles_m * sd.tiles_n;
    const int split = (int)(tile / ntile);
    const int64_t t2 = tile - (int64_t)split * ntile;
    const int64_t m0 = (t2 % sd.tiles_m) * BM, n0 = (t2 / sd.tiles_m) * BN;
    const int64_t M = sd.M, N = sd.N, K = sd.K;
    const T *__restrict__ A = (const T *)sd.a;
    const T *__restrict__ B = (const T *)sd.b;
    const int64_t *__restrict__ offAK = sd.offAK;
    const int64_t *__restrict__ offBK = sd.offBK;
    const int64_t ap = sd.a_plane, bp = sd.b_plane;
    // contracted range of this CTA, in k-tiles
    const int64_t nkt_all = (K + BK - 1) / BK;
    const int64_t kt0 = (int64_t)split * sd.ktiles_per_split;
    const int64_t kt1 = min(nkt_all, kt0 + (int64_t)sd.ktiles_per_split);
    const int nkt = kt1 > kt0 ? (int)(kt1 - kt0) : 0;

    if (sd.part == nullptr)
        for (int i = tid; i < BM + BN; i += NT) {
            if (i < BM) sCM[i] = (m0 + i < M) ? sd.offCM[m0 + i] : 0;
            else sCN[i - BM] = (n0 + i - BM < N) ? sd.offCN[n0 + i - BM] : 0;
        }

    // this thread's share of the A and B tiles
    int aK[LA], aS[LA], bK[LB], bS[LB];   // k within the tile, shared-row offset
    int64_t aOff[LA], bOff[LB];
    bool aOk[LA], bOk[LB];
#pragma unroll
    for (int i = 0; i < LA; ++i) {
        const int e = tid + i * NT;
        const int mi = amf ? e % BM : e / BK;
        aK[i] = amf ? e / BM : e % BK;
        aS[i] = aK[i] * RA + mi;
        aOk[i] = m0 + mi < M;
        aOff[i] = aOk[i] ? sd.offAM[m0 + mi] : 0;
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
        const int e = tid + i * NT;
        const int ni = bnf ? e % BN : e / BK;
        bK[i] = bnf ? e / BN : e % BK;
        bS[i] = bK[i] * RB + ni;
        bOk[i] = n0 + ni < N;
        bOff[i] = bOk[i] ? sd.offBN[n0 + ni] : 0;
    }

    // offsets of the contracted indices of a k-tile, one tile ahead
    int64_t kA[LA], kB[LB];
    auto load_koff = [&](int t) {   // t: local k-tile index
        const int64_t kb = (kt0 + t) * BK;
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            const int64_t k = kb + aK[i];
            kA[i] = (t < nkt && k < K) ? __ldg(offAK + k) : -1;
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const int64_t k = kb + bK[i];
            kB[i] = (t < nkt && k < K) ? __ldg(offBK + k) : -1;
        }
    };
    auto issue = [&](int st) {      // cp.async of the tile whose offsets are in kA/kB
        T *a0 = As + st * 2 * PA, *b0 = Bs + st * 2 * PB;
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            const bool v = aOk[i] && kA[i] >= 0;
            const T *src = v ? A + aOff[i] + kA[i] : A;
            cp_async_el(a0 + aS[i], src, sizeof(T), v);
            cp_async_el(a0 + PA + aS[i], v ? src + ap : A, sizeof(T), v);
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const bool v = bOk[i] && kB[i] >= 0;
            const T *src = v ? B + bOff[i] + kB[i] : B;
            cp_async_el(b0 + bS[i], src, sizeof(T), v);
            cp_async_el(b0 + PB + bS[i], v ? src + bp : B, sizeof(T), v);
        }
    };

    const int ty = tid / Cfg::TXN, tx = tid % Cfg::TXN;
    T cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0;

    grid_dep_wait();   // operands may be the previous kernel's results
    // prologue: tiles 0 .. STAGES-2 in flight, offsets of tile STAGES-1 loaded
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        load_koff(s);
        if (s < nkt) issue(s);
        cp_async_commit();
    }
    load_koff(STAGES - 1);

    // one k row of this thread's A and B fragments from shared memory
    auto frag = [&](const T *a0, const T *b0, int kk, T *xr, T *xi, T *yr, T *yi) {
#pragma unroll
        for (int v = 0; v < Cfg::VA; ++v) {
            V r = *reinterpret_cast<const V *>(a0 + kk * RA + v * Vec16<T>::n);
            V q = *reinterpret_cast<const V *>(a0 + PA + kk * RA + v * Vec16<T>::n);
            const T *rr = reinterpret_cast<const T *>(&r), *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int u = 0; u < Vec16<T>::n; ++u) {
                xr[v * Vec16<T>::n + u] = rr[u];
                xi[v * Vec16<T>::n + u] = qq[u];
            }
        }
#pragma unroll
        for (int v = 0; v < Cfg::VB; ++v) {
            V r = *reinterpret_cast<const V *>(b0 + kk * RB + v * Vec16<T>::n);
            V q = *reinterpret_cast<const V *>(b0 + PB + kk * RB + v * Vec16<T>::n);
            const T *rr = reinterpret_cast<const T *>(&r), *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int u = 0; u < Vec16<T>::n; ++u) {
                yr[v * Vec16<T>::n + u] = rr[u];
                yi[v * Vec16<T>::n + u] = qq[u];
            }
        }
    };
    auto macs = [&](const T *xr, const T *xi, const T *yr, const T *yi) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) cmac(cr[i][j], ci[i][j], xr[i], xi[i], yr[j], yi[j]);
    };

    for (int kt = 0; kt < nkt; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();   // tile kt visible to all; stage of tile kt-1 free
        if (kt + STAGES - 1 < nkt) issue((kt + STAGES - 1) % STAGES);
        cp_async_commit();
        load_koff(kt + STAGES);
        const int st = kt % STAGES;
        const T *a0 = As + st * 2 * PA + ty * TM;
        const T *b0 = Bs + st * 2 * PB + tx * TN;
        // two register fragments: row kk+1 is read from shared memory while
        // the products of row kk issue; the loop is unrolled only KU times so
        // that the body stays within the instruction cache
        constexpr int kKU = ROSNET_TILED_KU;
        T xr0[TM], xi0[TM], yr0[TN], yi0[TN], xr1[TM], xi1[TM], yr1[TN], yi1[TN];
        frag(a0, b0, 0, xr0, xi0, yr0, yi0);
#pragma unroll(kKU)
        for (int kk = 0; kk < BK; kk += 2) {
            frag(a0, b0, kk + 1, xr1, xi1, yr1, yi1);
            macs(xr0, xi0, yr0, yi0);
            if (kk + 2 < BK) frag(a0, b0, kk + 2, xr0, xi0, yr0, yi0);
            macs(xr1, xi1, yr1, yi1);
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // every warp is done with the ring: it holds the output tile now

    store_tile<T, BM, BN, TM, TN>(sd, cr, ci, As, sCM, sCN, m0, n0, split, ty, tx);
}

// Short contraction ranges: each CTA gathers its whole A (BM x Kc) and B
// (Kc x BN) tiles into shared memory in one pass -- every thread's loads
// issued before any is used, coalesced along each operand's unit-stride
// digit, offsets read from shared copies of the offset tables -- then runs
// the Kc loop from shared memory.  Kc <= kDirectK: the whole K, or with a
// split one kDirectK-long slice of it per CTA (partials summed by
// gett_reduce_kernel).  No staging ring, small code: for contractions whose
// per-CTA range is too short to fill a pipeline.
template <typename T, int BM_, int BN_>
struct DirectCfg {
    static constexpr int BM = BM_, BN = BN_, KM = kDirectK;
    static constexpr int TN = 4, TXN = BN / TN, TY = 256 / TXN, TM = BM / TY;   // 4 columns per thread
    static constexpr int PAD = 16 / (int)sizeof(T);
    static constexpr int RA = BM + PAD, RB = BN + PAD;
    static constexpr int NEA = BM * KM / 256, NEB = BN * KM / 256;   // elements per thread
    static constexpr size_t smem = sizeof(T) * 2 * (size_t)KM * (RA + RB);
    static_assert(TXN * TY == 256 && TM * TY == BM && TM % 4 == 0 && NEB >= 1, "tile shape");
    static_assert((size_t)(BM + 1) * (BN + 1) * sizeof(T) <= smem, "epilogue staging exceeds the tiles");
};

template <typename T, int BM, int BN, bool amf, bool bnf>
__device__ __forceinline__ void direct_body(const GettDesc &sd, T *As, T *Bs, int64_t *sAM, int64_t *sBN,
                                            int64_t *sAK, int64_t *sBK, int64_t *sCM, int64_t *sCN) {
    using Cfg = DirectCfg<T, BM, BN>;
    using V = typename Vec16<T>::type;
    constexpr int KM = Cfg::KM, TM = Cfg::TM, TN = Cfg::TN, TXN = Cfg::TXN;
    constexpr int RA = Cfg::RA, RB = Cfg::RB, NEA = Cfg::NEA, NEB = Cfg::NEB;
    const int tid = threadIdx.x;
    const int64_t t = (int64_t)blockIdx.x - sd.tile_begin;
    const int64_t ntile = sd.tiles_m * sd.tiles_n;
    const int split = (int)(t / ntile);
    const int64_t t2 = t - (int64_t)split * ntile;
    const int64_t m0 = (t2 % sd.tiles_m) * BM, n0 = (t2 / sd.tiles_m) * BN;
    const int64_t M = sd.M, N = sd.N;
    const int64_t k0 = (int64_t)split * KM;
    const int K = (int)min((int64_t)KM, sd.K - k0);   // this CTA's contracted range
    // offsets of this tile's rows / columns / contracted indices (static tables)
    for (int i = tid; i < BM + BN + 2 * KM; i += 256) {
        if (i < BM) {
            sAM[i] = m0 + i < M ? sd.offAM[m0 + i] : -1;
            sCM[i] = m0 + i < M ? sd.offCM[m0 + i] : 0;
        } else if (i < BM + BN) {
            const int j = i - BM;
            sBN[j] = n0 + j < N ? sd.offBN[n0 + j] : -1;
            sCN[j] = n0 + j < N ? sd.offCN[n0 + j] : 0;
        } else if (i < BM + BN + KM) {
            const int k = i - BM - BN;
            sAK[k] = k < K ? sd.offAK[k0 + k] : 0;
        } else {
            const int k = i - BM - BN - KM;
            sBK[k] = k < K ? sd.offBK[k0 + k] : 0;
        }
    }
    __syncthreads();
    grid_dep_wait();   // operands may be the previous kernel's results
    const T *__restrict__ A = (const T *)sd.a;
    const T *__restrict__ B = (const T *)sd.b;
    const int64_t ap = sd.a_plane, bp = sd.b_plane;
    // loads in flight together, at most GA elements of A (and all of B, in the
    // first batch) per thread at a time
    constexpr int GA = NEA < 16 ? NEA : 16;
#pragma unroll 1
    for (int j0 = 0; j0 < NEA; j0 += GA) {
        T ar[GA], ai[GA], br[NEB], bi[NEB];
#pragma unroll
        for (int j = 0; j < GA; ++j) {
            const int e = tid + 256 * (j0 + j);
            const int am = amf ? e % BM : e / KM, ak = amf ? e / BM : e % KM;
            const int64_t oa = (ak < K && sAM[am] >= 0) ? sAM[am] + sAK[ak] : -1;
            ar[j] = oa >= 0 ? A[oa] : T(0);
            ai[j] = oa >= 0 ? A[oa + ap] : T(0);
        }
        if (j0 == 0) {
#pragma unroll
            for (int j = 0; j < NEB; ++j) {
                const int e = tid + 256 * j;
                const int bn = bnf ? e % BN : e / KM, bk = bnf ? e / BN : e % KM;
                const int64_t ob = (bk < K && sBN[bn] >= 0) ? sBN[bn] + sBK[bk] : -1;
                br[j] = ob >= 0 ? B[ob] : T(0);
                bi[j] = ob >= 0 ? B[ob + bp] : T(0);
            }
#pragma unroll
            for (int j = 0; j < NEB; ++j) {
                const int e = tid + 256 * j;
                const int bn = bnf ? e % BN : e / KM, bk = bnf ? e / BN : e % KM;
                Bs[bk * RB + bn] = br[j];
                Bs[KM * RB + bk * RB + bn] = bi[j];
            }
        }
#pragma unroll
        for (int j = 0; j < GA; ++j) {
            const int e = tid + 256 * (j0 + j);
            const int am = amf ? e % BM : e / KM, ak = amf ? e / BM : e % KM;
            As[ak * RA + am] = ar[j];
            As[KM * RA + ak * RA + am] = ai[j];
        }
    }
    __syncthreads();
    const int ty = tid / TXN, tx = tid % TXN;
    T cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0;
    const T *a0 = As + ty * TM, *b0 = Bs + tx * TN;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        T xr[TM], xi[TM], yr[TN], yi[TN];
#pragma unroll
        for (int v = 0; v < TM * (int)sizeof(T) / 16; ++v) {
            const V r = *reinterpret_cast<const V *>(a0 + k * RA + v * Vec16<T>::n);
            const V q = *reinterpret_cast<const V *>(a0 + KM * RA + k * RA + v * Vec16<T>::n);
            const T *rr = reinterpret_cast<const T *>(&r), *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int u = 0; u < Vec16<T>::n; ++u) {
                xr[v * Vec16<T>::n + u] = rr[u];
                xi[v * Vec16<T>::n + u] = qq[u];
            }
        }
#pragma unroll
        for (int v = 0; v < TN * (int)sizeof(T) / 16; ++v) {
            const V r = *reinterpret_cast<const V *>(b0 + k * RB + v * Vec16<T>::n);
            const V q = *reinterpret_cast<const V *>(b0 + KM * RB + k * RB + v * Vec16<T>::n);
            const T *rr = reinterpret_cast<const T *>(&r), *qq = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int u = 0; u < Vec16<T>::n; ++u) {
                yr[v * Vec16<T>::n + u] = rr[u];
                yi[v * Vec16<T>::n + u] = qq[u];
            }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) cmac(cr[i][j], ci[i][j], xr[i], xi[i], yr[j], yi[j]);
    }
    __syncthreads();   // the operand tiles become the output staging area
    store_tile<T, BM, BN, TM, TN>(sd, cr, ci, As, sCM, sCN, m0, n0, split, ty, tx);
}

template <typename T, int BM, int BN>
__global__ void __launch_bounds__(256) gett_direct_kernel(const __grid_constant__ GroupArgs g) {
    using Cfg = DirectCfg<T, BM, BN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);          // [2 planes][KM][RA]
    T *Bs = As + 2 * Cfg::KM * Cfg::RA;                // [2 planes][KM][RB]
    __shared__ GettDesc sd;
    __shared__ int64_t sAM[BM], sBN[BN], sAK[Cfg::KM], sBK[Cfg::KM], sCM[BM], sCN[BN];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    switch (((sd.flags & kFlagAMFast) ? 2 : 0) | ((sd.flags & kFlagBNFast) ? 1 : 0)) {
        case 0: direct_body<T, BM, BN, false, false>(sd, As, Bs, sAM, sBN, sAK, sBK, sCM, sCN); break;
        case 1: direct_body<T, BM, BN, false, true>(sd, As, Bs, sAM, sBN, sAK, sBK, sCM, sCN); break;
        case 2: direct_body<T, BM, BN, true, false>(sd, As, Bs, sAM, sBN, sAK, sBK, sCM, sCN); break;
        default: direct_body<T, BM, BN, true, true>(sd, As, Bs, sAM, sBN, sAK, sBK, sCM, sCN); break;
    }
}

template <typename T, int BM, int BN, int BK, int STAGES>
__global__ void __launch_bounds__(256, (TiledCfg<T, BM, BN, BK, STAGES>::TM == 4 && TiledCfg<T, BM, BN, BK, STAGES>::LA <= 4 && sizeof(T) == 4) ? ROSNET_TILED_MINB : 1)
    gett_tiled_kernel(const __grid_constant__ GroupArgs g) {
    using Cfg = TiledCfg<T, BM, BN, BK, STAGES>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);                  // [STAGES][2 planes][BK][RA]
    T *Bs = As + STAGES * 2 * BK * Cfg::RA;                     // [STAGES][2 planes][BK][RB]
    __shared__ GettDesc sd;
    __shared__ int64_t sCM[BM], sCN[BN];
    grid_dep_launch();
    if (threadIdx.x < 32) load_desc(g, sd);
    __syncthreads();
    switch (((sd.flags & kFlagAMFast) ? 2 : 0) | ((sd.flags & kFlagBNFast) ? 1 : 0)) {
        case 0: tiled_body<T, BM, BN, BK, STAGES, false, false>(sd, As, Bs, sCM, sCN); break;
        case 1: tiled_body<T, BM, BN, BK, STAGES, false, true>(sd, As, Bs, sCM, sCN); break;
        case 2: tiled_body<T, BM, BN, BK, STAGES, true, false>(sd, As, Bs, sCM, sCN); break;
        default: tiled_body<T, BM, BN, BK, STAGES, true, true>(sd, As, Bs, sCM, sCN); break;
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
// C^T = B^T A^T: exchange the roles of the two operands (no data moves).
static void swap_operands(GettDesc &d) {
    std::swap(d.offAM, d.offBN);
    std::swap(d.offCM, d.offCN);
    std::swap(d.offAK, d.offBK);
    std::swap(d.M, d.N);
    int f = d.flags;
    d.flags = ((f & kFlagAMFast) ? kFlagBNFast : 0) | ((f & kFlagBNFast) ? kFlagAMFast : 0) |
              ((f & kFlagCNFast) ? 0 : kFlagCNFast) | ((f & kFlagSwapped) ? 0 : kFlagSwapped) |
              ((f & kFlagADense) ? kFlagBDense : 0) | ((f & kFlagBDense) ? kFlagADense : 0) |
              ((f & kFlagAMVec) ? kFlagBNVec : 0) | ((f & kFlagBNVec) ? kFlagAMVec : 0) |
              ((f & kFlagCMVec) ? kFlagCNVec : 0) | ((f & kFlagCNVec) ? kFlagCMVec : 0) |
              ((f & kFlagCNInner) ? kFlagCMInner : 0) | ((f & kFlagCMInner) ? kFlagCNInner : 0) |
              (f & kFlagAtomic);
}

constexpr int kTiledStages = 3;

bool tc_mode_of(int precision, int *mode);
int tc_tile_m();
int tc_tile_n();
void f32p_tile(int64_t N, int *bm, int *bn);
int64_t f32p_skinny_split(const GettDesc &d);
void f32p_set_geometry(GettDesc &d);
size_t tc_workspace_bytes(const GettDesc &d, int mode);
size_t tc_workspace_bytes_bound(const GettDesc &d, int mode);
void tc_workspace_clear(const GettDesc &d, int mode, void *ws, cudaStream_t s);
bool f32p_stream_k_pays(const GettDesc &d, int reduce_mode);
bool f32p_stream_k_worth_timing(const GettDesc &d, int reduce_mode);
void launch_tc_problem(int mode, const GettDesc &d, const GroupArgs &ga, void *ws, cudaStream_t s,
                       bool pack_a, bool pack_b, const std::function<void()> &before_gemm = {},
                       bool pdl = true);

// The CTAs a gate problem launches at most.  For the looping kinds (a side
// of 4: at most two CTAs fit on an SM), as many as are resident at once,
// each looping over its runs of rows (measured on [2]^28: 0.72 -> 0.87 of the
// HBM copy rate for a two-qubit gate); for the others one CTA per 256 runs,
// which keeps more loads in flight for the one-qubit gates (0.87 / 0.94
// against 0.79 / 0.85 looping).
static int64_t gate_resident_ctas(int kind) {
    static std::atomic<int64_t> cache[9];
    const int i = kind - kKindGateBase;
    const int64_t c = cache[i].load(std::memory_order_relaxed);
    if (c) return c;
    const void *fn = nullptr;
    switch (i) {
        case 0: fn = (const void *)gett_gate_kernel<1, 1>; break;
        case 1: fn = (const void *)gett_gate_kernel<1, 2>; break;
        case 2: fn = (const void *)gett_gate_kernel<1, 4>; break;
        case 3: fn = (const void *)gett_gate_kernel<2, 1>; break;
        case 4: fn = (const void *)gett_gate_kernel<2, 2>; break;
        case 5: fn = (const void *)gett_gate_kernel<2, 4>; break;
        case 6: fn = (const void *)gett_gate_kernel<4, 1>; break;
        case 7: fn = (const void *)gett_gate_kernel<4, 2>; break;
        default: fn = (const void *)gett_gate_kernel<4, 4>; break;
    }
    const int lk = i / 3, ln = i % 3;   // log2 K, log2 N
    if (!gate_loops(1 << lk, 1 << ln)) {
        cache[i].store(int64_t(1) << 40, std::memory_order_relaxed);
        return int64_t(1) << 40;
    }
    int per = 0;
    RN_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, 0));
    const int64_t v = (int64_t)std::max(per, 1) * num_sms();
    cache[i].store(v, std::memory_order_relaxed);
    return v;
}

void choose_kernel(GettDesc &d, int dtype, int precision, int reduce_mode) {
    const int64_t kSMs = num_sms();
    d.ksplit = 1;
    d.ktiles_per_split = 0x7fffffff;
    d.part = nullptr;
    const int64_t MN = d.M * d.N;
    int tcmode;
    if (dtype == ROSNET_C64 && tc_mode_of(precision, &tcmode) && std::max(d.M, d.N) >= 128 &&
        std::min(d.M, d.N) >= 64 && d.K >= 32) {
        if (d.N > d.M) swap_operands(d);
        d.kind = kKindTcTF32 + tcmode;
        d.tiles_m = (d.M + tc_tile_m() - 1) / tc_tile_m();
        d.tiles_n = (d.N + tc_tile_n() - 1) / tc_tile_n();
        return;
    }
    // low arithmetic intensity: a large operand against at most 4 x 4 entries
    // (a gate on some axes of a big tensor, a projection): streamed once with
    // vector accesses, when the layouts allow them
    if (dtype == ROSNET_C64 && gate_log2(d.K) >= 0 && gate_log2(std::min(d.M, d.N)) >= 0 &&
        std::max(d.M, d.N) >= 2048) {
        GettDesc e = d;
        if (e.N > e.M) swap_operands(e);
        if ((e.flags & kFlagAMVec) && (e.flags & (kFlagCMVec | kFlagCNInner))) {
            d = e;
            d.kind = kKindGateBase + 3 * gate_log2(d.K) + gate_log2(d.N);
            d.tiles_m = std::min<int64_t>((d.M + 256 * gate_rows(d.kind) - 1) / (256 * gate_rows(d.kind)),
                                          gate_resident_ctas(d.kind));
            d.tiles_n = 1;
            return;
        }
    }
    // large FP32 contractions: pack once, then TMA-fed FFMA tiles (no split-K).
    // Short contractions (32 <= K < 128) only when both operands are read in
    // place: a pack pass would cost more than the one or few k-tiles it feeds
    const bool in_place = (d.flags & kFlagADense) && (d.flags & kFlagBDense);
    if (dtype == ROSNET_C64 && reduce_mode != kReduceTree && reduce_mode != kReduceCommutative &&
        std::min(d.M, d.N) >= 64 && (d.K >= 128 || (d.K >= 32 && in_place)) &&
        8.0 * (double)MN * (double)d.K >= 268435456.0) {
        const int64_t t = ((d.M + 63) / 64) * ((d.N + 63) / 64);
        if (t >= 120) {
            if (d.N > d.M) swap_operands(d);
            d.kind = kKindPackF32;
            d.tiles_m = (d.M + 63) / 64;
            d.tiles_n = (d.N + 63) / 64;
            if (f32p_stream_k_pays(d, reduce_mode)) d.flags |= kFlagStreamK;
            return;
        }
    }
    // few columns and a long contraction (e.g. 256 x 16 x 4096): the same
    // GEMM with 128 x 16 tiles and the contraction split over CTAs, its
    // partial results summed in split order
    if (dtype == ROSNET_C64 && (reduce_mode == kReduceAuto || reduce_mode == kReduceTree) &&
        std::min(d.M, d.N) <= 16 && std::max(d.M, d.N) >= 128 && d.K >= 512 &&
        8.0 * (double)MN * (double)d.K >= 67108864.0) {
        if (d.N > d.M) swap_operands(d);
        d.kind = kKindPackF32;
        f32p_set_geometry(d);
        return;
    }
    // short contractions: whole tiles in one pass
    if (d.K >= 8 && d.K <= kDirectK && std::min(d.M, d.N) >= 16 && MN >= 4096) {
        if (d.N > d.M) swap_operands(d);
        d.kind = kKindDirect;
        d.tiles_m = (d.M + 63) / 64;
        d.tiles_n = (d.N + 63) / 64;
        return;
    }
    const bool tiled_ok = d.K >= 16 && std::min(d.M, d.N) >= 16 && MN >= 2048;
    if (tiled_ok) {
        if (d.N > d.M) swap_operands(d);   // the BM side takes the larger extent
        // few columns: narrow tiles; else 128x64 when both sides are large
        int kind = kKindTiled;
        if (d.N <= 16 && d.M >= 256 && tiled_kind_ok(kKindTiled256x16, dtype, d.M, d.N)) kind = kKindTiled256x16;
        else if (d.N <= 32 && d.M >= 128 && tiled_kind_ok(kKindTiled128x32, dtype, d.M, d.N)) kind = kKindTiled128x32;
        else if (tiled_kind_ok(kKindTiledWide, dtype, d.M, d.N)) kind = kKindTiledWide;
        int BM, BN;
        tiled_tile(kind, &BM, &BN);
        const int BK = dtype == ROSNET_C64 ? 16 : 8;
        d.kind = kind;
        d.tiles_m = (d.M + BM - 1) / BM;
        d.tiles_n = (d.N + BN - 1) / BN;
        // split the contracted range when the tile grid cannot fill the GPU
        // (or when asked to), unless the sequential reduction is requested
        const int64_t tiles = d.tiles_m * d.tiles_n;
        const int64_t nkt = (d.K + BK - 1) / BK;
        const bool forced = reduce_mode == kReduceTree || reduce_mode == kReduceCommutative;
        // FP64 runs at a small fraction of the FP32 rate on this GPU (a few
        // DFMA per clock per SM), so even one k-tile of a 64 x 64 tile keeps a
        // CTA busy far longer than its prologue: complex128 problems split
        // down to single k-tiles to occupy every SM
        const bool fp64 = dtype == ROSNET_C128;
        if (reduce_mode != kReduceSequential &&
            ((tiles < kSMs && (nkt >= 32 || (fp64 && nkt >= 2))) || (forced && nkt >= 2))) {
            int64_t want = std::max<int64_t>((2 * kSMs + tiles - 1) / tiles, forced ? 2 : 1);
            // auto: at least 8 k-tiles per range (complex64), 1 (complex128)
            int64_t cap = (forced || fp64) ? nkt : nkt / 8;
            int64_t ks = std::max<int64_t>(1, std::min<int64_t>(std::min(want, cap), 64));
            if (ks > 1) {
                d.ktiles_per_split = (int)((nkt + ks - 1) / ks);
                d.ksplit = (int)((nkt + d.ktiles_per_split - 1) / d.ktiles_per_split);
                if (reduce_mode == kReduceCommutative) d.flags |= kFlagAtomic;
            }
        }
        return;
    }
    if (d.K >= 1024 && MN <= 256) {
        d.kind = kKindDot;
        d.tiles_m = MN;
        d.tiles_n = kDotCTAs;   // one cluster per output
    } else if (d.K >= 128 && MN <= (int64_t(1) << 16)) {
        d.kind = kKindWarpK;
        d.tiles_m = (MN + 7) / 8;
        d.tiles_n = 1;
    } else {
        d.kind = kKindSmall;
        d.tiles_m = (MN + 255) / 256;
        d.tiles_n = 1;
    }
}

int gate_record_class(const GettView &v, int dtype, int precision, int reduce_mode, int clear_flags) {
    GettDesc t;
    memset(&t, 0, sizeof(t));
    fill_desc_tables(t, v, nullptr, nullptr, nullptr);
    t.flags &= ~clear_flags;
    choose_kernel(t, dtype, precision, reduce_mode);
    if (!is_gate_kind(t.kind)) return -1;
    return (t.flags & kFlagSwapped) ? 1 : 0;   // the kernel walks the larger class as its M
}

size_t desc_part_bytes(const GettDesc &d, int dtype) {
    if (d.ksplit <= 1 || (d.flags & kFlagAtomic)) return 0;
    return (size_t)d.ksplit * 2 * (size_t)(d.M * d.N) * (dtype == ROSNET_C64 ? 4 : 8);
}

template <typename T, int BM, int BN>
static void launch_direct(dim3 grid, const GroupArgs &ga, cudaStream_t s, bool pdl) {
    using Cfg = DirectCfg<T, BM, BN>;
    static std::atomic<uint64_t> done{0};   // once per device
    uint64_t bit;
    if (!attrs_set(done, &bit)) {
        RN_CHECK_CUDA(cudaFuncSetAttribute(gett_direct_kernel<T, BM, BN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem));
        done.fetch_or(bit, std::memory_order_release);
    }
    launch_pdl(gett_direct_kernel<T, BM, BN>, grid, 256, Cfg::smem, s, pdl, ga);
}

template <typename T, int BM, int BN, int BK>
static void launch_tiled(dim3 grid, const GroupArgs &ga, cudaStream_t s, bool pdl) {
    using Cfg = TiledCfg<T, BM, BN, BK, kTiledStages>;
    static std::atomic<uint64_t> done{0};   // once per device
    uint64_t bit;
    if (!attrs_set(done, &bit)) {
        RN_CHECK_CUDA(cudaFuncSetAttribute(gett_tiled_kernel<T, BM, BN, BK, kTiledStages>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem));
        done.fetch_or(bit, std::memory_order_release);
    }
    launch_pdl(gett_tiled_kernel<T, BM, BN, BK, kTiledStages>, grid, 256, Cfg::smem, s, pdl, ga);
}

static void launch_group_args(int kind, int dtype, const GroupArgs &ga, int64_t total_ctas,
                              cudaStream_t s, bool pdl = true) {
    if (total_ctas <= 0) return;
    if (total_ctas > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "too many tiles in one launch");
    dim3 grid((unsigned)total_ctas);
    if (is_packed_kind(kind))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "tensor-core problems are launched with their workspace");
    if (is_gate_kind(kind)) {
        if (dtype != ROSNET_C64) RN_FAIL(ROSNET_ERR_INVALID_ARG, "the gate kernel is complex64 only");
        switch (kind - kKindGateBase) {
            case 0: launch_pdl(gett_gate_kernel<1, 1>, grid, 256, 0, s, pdl, ga); break;
            case 1: launch_pdl(gett_gate_kernel<1, 2>, grid, 256, 0, s, pdl, ga); break;
            case 2: launch_pdl(gett_gate_kernel<1, 4>, grid, 256, 0, s, pdl, ga); break;
            case 3: launch_pdl(gett_gate_kernel<2, 1>, grid, 256, 0, s, pdl, ga); break;
            case 4: launch_pdl(gett_gate_kernel<2, 2>, grid, 256, 0, s, pdl, ga); break;
            case 5: launch_pdl(gett_gate_kernel<2, 4>, grid, 256, 0, s, pdl, ga); break;
            case 6: launch_pdl(gett_gate_kernel<4, 1>, grid, 256, 0, s, pdl, ga); break;
            case 7: launch_pdl(gett_gate_kernel<4, 2>, grid, 256, 0, s, pdl, ga); break;
            default: launch_pdl(gett_gate_kernel<4, 4>, grid, 256, 0, s, pdl, ga); break;
        }
        g_launches++;
        RN_CHECK_CUDA(cudaGetLastError());
        return;
    }
    if (dtype == ROSNET_C64) {
        switch (kind) {
            case kKindSmall: launch_pdl(gett_small_kernel<float>, grid, 256, 0, s, pdl, ga); break;
            case kKindWarpK: launch_pdl(gett_warpk_kernel<float>, grid, 256, 0, s, pdl, ga); break;
            case kKindReduce: launch_pdl(gett_reduce_kernel<float>, grid, 256, 0, s, pdl, ga); break;
            case kKindZero: launch_pdl(gett_zero_kernel<float>, grid, 256, 0, s, pdl, ga); break;
            case kKindDot: launch_pdl(gett_dot_kernel<float>, grid, 256, 0, s, pdl, ga); break;
            case kKindTiledWide: launch_tiled<float, 128, 64, 16>(grid, ga, s, pdl); break;
            case kKindTiled256x16: launch_tiled<float, 256, 16, 16>(grid, ga, s, pdl); break;
            case kKindDirect: launch_direct<float, 64, 64>(grid, ga, s, pdl); break;
            case kKindDirect256x16: launch_direct<float, 256, 16>(grid, ga, s, pdl); break;
            case kKindTiled128x32: launch_tiled<float, 128, 32, 16>(grid, ga, s, pdl); break;
            default: launch_tiled<float, 64, 64, 16>(grid, ga, s, pdl); break;
        }
    } else {
        switch (kind) {
            case kKindSmall: launch_pdl(gett_small_kernel<double>, grid, 256, 0, s, pdl, ga); break;
            case kKindWarpK: launch_pdl(gett_warpk_kernel<double>, grid, 256, 0, s, pdl, ga); break;
            case kKindReduce: launch_pdl(gett_reduce_kernel<double>, grid, 256, 0, s, pdl, ga); break;
            case kKindZero: launch_pdl(gett_zero_kernel<double>, grid, 256, 0, s, pdl, ga); break;
            case kKindDot: launch_pdl(gett_dot_kernel<double>, grid, 256, 0, s, pdl, ga); break;
            case kKindDirect: launch_direct<double, 64, 64>(grid, ga, s, pdl); break;
            default: launch_tiled<double, 64, 64, 8>(grid, ga, s, pdl); break;
        }
    }
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

void launch_forest(int dtype, const GettDesc *descs, const int64_t *prog, int64_t ctas, cudaStream_t s) {
    if (ctas <= 0) return;
    if (ctas > 0x7fffffffLL) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "too many groups in one launch");
    if (dtype == ROSNET_C64)
        launch_pdl(gett_forest_kernel<float>, dim3((unsigned)ctas), kForestThreads, 0, s, true, descs, prog);
    else
        launch_pdl(gett_forest_kernel<double>, dim3((unsigned)ctas), kForestThreads, 0, s, true, descs, prog);
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

void launch_gett_group(int kind, int dtype, const GettDesc *descs, int ndesc, int64_t total_ctas,
                       cudaStream_t s) {
    GroupArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.descs = descs;
    ga.ndesc = ndesc;
    launch_group_args(kind, dtype, ga, total_ctas, s);
}

static void launch_gett_single(const GettDesc &d, int kind, int64_t ctas, int dtype, cudaStream_t s,
                               bool pdl = true) {
    GroupArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.descs = nullptr;
    ga.ndesc = 1;
    ga.single = d;
    ga.single.tile_begin = 0;
    launch_group_args(kind, dtype, ga, ctas, s, pdl);
}

// ---------------------------------------------------------------------------
// autotuner: candidate tile shapes and contracted-range splits, timed
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
    int dtype, flags;
    int64_t M, N, K;
    bool operator==(const TuneKey &o) const {
        return dtype == o.dtype && flags == o.flags && M == o.M && N == o.N && K == o.K;
    }
};
struct TuneKeyHash {
    size_t operator()(const TuneKey &k) const {
        return (size_t)(k.M * 1000003 ^ k.N * 10007 ^ k.K * 101 ^ k.flags * 7 ^ k.dtype);
    }
};
struct TuneChoice { int kind; int64_t tiles_m, tiles_n; int32_t ksplit, kps; int32_t flags; };
std::mutex g_tune_mu;
auto &g_tune = *new std::unordered_map<TuneKey, TuneChoice, TuneKeyHash>();

void apply_split(GettDesc &d, int BK, int64_t ks) {
    const int64_t nkt = (d.K + BK - 1) / BK;
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, std::min<int64_t>(nkt, 64)));
    d.ktiles_per_split = ks > 1 ? (int)((nkt + ks - 1) / ks) : 0x7fffffff;
    d.ksplit = ks > 1 ? (int)((nkt + d.ktiles_per_split - 1) / d.ktiles_per_split) : 1;
}
// Direct kinds split K into kDirectK-long slices, one per CTA (ktiles_per_split
// counts slices); false when the partial sums would exceed 2^24 entries.
bool direct_split(GettDesc &d) {
    const int64_t ks = (d.K + kDirectK - 1) / kDirectK;
    if (ks > 1 && (double)ks * (double)d.M * (double)d.N > (double)(1 << 24)) return false;
    d.ksplit = (int)std::max<int64_t>(ks, 1);
    d.ktiles_per_split = ks > 1 ? 1 : 0x7fffffff;
    return true;
}
}  // namespace

// Tile grid and contraction split of the TMA-fed FP32 GEMM for d's shape
// (N <= M): 64 x 64 tiles, one CTA per tile; or for few columns 128 x 16
// tiles with the contraction split (ktiles_per_split in 32-deep k-tiles).
void f32p_set_geometry(GettDesc &d) {
    int bm, bn;
    f32p_tile(d.N, &bm, &bn);
    d.tiles_m = (d.M + bm - 1) / bm;
    d.tiles_n = (d.N + bn - 1) / bn;
    const int64_t ks = f32p_skinny_split(d);
    apply_split(d, 32, ks > 0 ? ks : 1);
}

int64_t reduce_ctas(const GettDesc &d);

// Time the candidate kernels of a CUDA-core problem (operands a, b; output
// written to c_scratch; split partials and packed operands to temporary
// workspaces) and keep the fastest in d: 64x64 and 128x64 register tiles,
// each with several contracted-range splits, and -- for plain FP32 when no
// reduction mode is forced -- the packed path.  Results are cached by
// (dtype, M, N, K, layout flags).
void autotune_problem(GettDesc &d, int dtype, bool packed_ok, int reduce_mode, cudaStream_t s) {
    if (!is_tiled_kind(d.kind) && d.kind != kKindPackF32 && !is_direct_kind(d.kind)) return;
    if (d.flags & kFlagAtomic) return;
    packed_ok = packed_ok && dtype == ROSNET_C64;
    const bool sk_ok = reduce_mode != kReduceSequential;   // one CTA per tile when asked for
    const TuneKey key{dtype, d.flags | (packed_ok ? 1 << 30 : 0) | (sk_ok ? 0 : 1 << 29), d.M, d.N, d.K};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            const TuneChoice &c = it->second;
            d.kind = c.kind;
            d.tiles_m = c.tiles_m;
            d.tiles_n = c.tiles_n;
            d.ksplit = c.ksplit;
            d.ktiles_per_split = c.kps;
            d.flags = (d.flags & ~kFlagStreamK) | (d.kind == kKindPackF32 && sk_ok ? (c.flags & kFlagStreamK) : 0);
            return;
        }
    }
    const int BK = dtype == ROSNET_C64 ? 16 : 8;
    const int64_t kSMs = num_sms();
    std::vector<GettDesc> cands;
    // the split the heuristic would pick for a 64x64 tiling
    int64_t auto_split = (d.kind == kKindPackF32 || is_direct_kind(d.kind)) ? 1 : d.ksplit;
    if (d.kind == kKindPackF32 || is_direct_kind(d.kind)) {
        const int64_t tiles = ((d.M + 63) / 64) * ((d.N + 63) / 64), nkt = (d.K + BK - 1) / BK;
        if (tiles < kSMs && nkt >= 32) auto_split = std::min<int64_t>((2 * kSMs + tiles - 1) / tiles, nkt / 8);
    }
    for (int kind : {(int)kKindTiled, (int)kKindTiledWide, (int)kKindTiled256x16, (int)kKindTiled128x32}) {
        if (!tiled_kind_ok(kind, dtype, d.M, d.N)) continue;
        int BM, BN;
        tiled_tile(kind, &BM, &BN);
        GettDesc x = d;
        x.kind = kind;
        x.tiles_m = (d.M + BM - 1) / BM;
        x.tiles_n = (d.N + BN - 1) / BN;
        for (int64_t ks : {int64_t(1), auto_split, 2 * auto_split, 4 * auto_split}) {
            GettDesc y = x;
            apply_split(y, BK, ks);
            bool dup = false;
            for (auto &c : cands)
                dup |= c.kind == y.kind && c.ksplit == y.ksplit && c.ktiles_per_split == y.ktiles_per_split;
            if (!dup) cands.push_back(y);
        }
    }
    for (int kind : {(int)kKindDirect, (int)kKindDirect256x16}) {
        if (!direct_kind_ok(kind, dtype, d.M, d.N)) continue;
        GettDesc y = d;
        int bm, bn;
        direct_tile(kind, &bm, &bn);
        y.kind = kind;
        y.tiles_m = (d.M + bm - 1) / bm;
        y.tiles_n = (d.N + bn - 1) / bn;
        if (direct_split(y)) cands.push_back(y);
    }
    if (packed_ok) {
        GettDesc y = d;
        y.kind = kKindPackF32;
        y.flags &= ~kFlagStreamK;
        f32p_set_geometry(y);
        cands.push_back(y);   // one CTA per tile (a split contraction for few columns)
        y.flags |= kFlagStreamK;
        // and stream-K wherever the tiles are few enough for its balance to
        // matter (timed: the heuristic's rule misses cases such as 2000 x 300
        // x 333, 160 tiles of 11 k-tiles: 1.36x)
        if (f32p_stream_k_worth_timing(y, reduce_mode)) cands.push_back(y);
    }
    for (GettDesc &c : cands)
        if (c.kind != kKindPackF32) c.flags &= ~kFlagStreamK;
    cudaEvent_t e0, e1;
    RN_CHECK_CUDA(cudaEventCreate(&e0));
    RN_CHECK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    GettDesc pick = d;
    for (GettDesc &c : cands) {
        const bool packed = c.kind == kKindPackF32;
        DevBuf part(packed ? 0 : desc_part_bytes(c, dtype), s);
        DevBuf ws(packed ? tc_workspace_bytes(c, kPackedModeF32) : 0, s);
        if (packed) tc_workspace_clear(c, kPackedModeF32, ws.p, s);
        c.part = part.p;
        GroupArgs ga;
        memset(&ga, 0, sizeof(ga));
        ga.ndesc = 1;
        ga.single = c;
        ga.single.tile_begin = 0;
        auto once = [&]() {
            if (packed) {
                launch_tc_problem(kPackedModeF32, c, ga, ws.p, s, true, true);
                return;
            }
            launch_gett_single(c, c.kind, desc_ctas(c), dtype, s);
            if (c.part) launch_gett_single(c, kKindReduce, reduce_ctas(c), dtype, s);
        };
        once();   // warm-up
        float ms = 1e30f;
        for (int trial = 0; trial < 3; ++trial) {   // best of three trials of 3 launches
            RN_CHECK_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) once();
            RN_CHECK_CUDA(cudaEventRecord(e1, s));
            RN_CHECK_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            RN_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        // the TMA-fed packed GEMM keeps its place unless another kernel is
        // clearly faster: timed back to back with its operands in L2, the
        // offset-table gathers of the tiled kernels look better than they do
        // inside a contraction (4096 x 256 x 256 in the 20-qubit amplitude:
        // within 3% here, 17% slower in place)
        const bool pick_packed = pick.kind == kKindPackF32;
        const float bar = packed == pick_packed ? best : packed ? best * 1.03f : best / 1.03f;
        if (ms < bar) {
            best = ms;
            pick = c;
        }
    }
    cudaEvent_t ev[2] = {e0, e1};
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    d.kind = pick.kind;
    d.tiles_m = pick.tiles_m;
    d.tiles_n = pick.tiles_n;
    d.ksplit = pick.ksplit;
    d.ktiles_per_split = pick.ktiles_per_split;
    d.flags = (d.flags & ~kFlagStreamK) | (pick.flags & kFlagStreamK);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = TuneChoice{d.kind, d.tiles_m, d.tiles_n, d.ksplit, d.ktiles_per_split, d.flags & kFlagStreamK};
}

// Geometry of a tuned choice for a problem of shape (M, N, K): tile grid
// and contracted-range split, as autotune_problem would have set them.
// False if the choice is not one the autotuner can make for that shape.
static bool tune_geometry(int dtype, int kind, int64_t M, int64_t N, int64_t K, int64_t ksplit,
                          TuneChoice *out) {
    if (M < 1 || N < 1 || K < 1 || ksplit < 1 || ksplit > (1 << 20)) return false;
    const int BK = dtype == ROSNET_C64 ? 16 : 8;
    GettDesc y;
    memset(&y, 0, sizeof(y));
    y.M = M;
    y.N = N;
    y.K = K;
    if (is_tiled_kind(kind) && tiled_kind_ok(kind, dtype, M, N)) {
        int BM, BN;
        tiled_tile(kind, &BM, &BN);
        y.tiles_m = (M + BM - 1) / BM;
        y.tiles_n = (N + BN - 1) / BN;
    } else if (is_direct_kind(kind) && direct_kind_ok(kind, dtype, M, N)) {
        int bm, bn;
        direct_tile(kind, &bm, &bn);
        y.tiles_m = (M + bm - 1) / bm;
        y.tiles_n = (N + bn - 1) / bn;
        if (!direct_split(y) || y.ksplit != ksplit) return false;
        *out = TuneChoice{kind, y.tiles_m, y.tiles_n, y.ksplit, y.ktiles_per_split, 0};
        return true;
    } else if (kind == kKindPackF32 && dtype == ROSNET_C64) {
        f32p_set_geometry(y);
        if (y.ksplit != ksplit) return false;   // its split is fixed by the shape
        *out = TuneChoice{kind, y.tiles_m, y.tiles_n, y.ksplit, y.ktiles_per_split, 0};
        return true;
    } else {
        return false;
    }
    apply_split(y, BK, ksplit);
    if (y.ksplit != ksplit) return false;   // not a split this shape can have
    *out = TuneChoice{kind, y.tiles_m, y.tiles_n, y.ksplit, y.ktiles_per_split, 0};
    return true;
}

// CTAs of the split-K reduction of a problem
int64_t reduce_ctas(const GettDesc &d) { return (d.M * d.N + 31) / 32; }

// ---------------------------------------------------------------------------
// one pairwise contraction
// ---------------------------------------------------------------------------
// The launches of one CUDA-core problem: C = 0 before an order-free split,
// the GEMM, the fixed-order sum of a stored split.  pdl applies to the first.
static void launch_sequence(const GettDesc &x, int dtype, cudaStream_t s, bool pdl) {
    if (x.flags & kFlagAtomic) {
        launch_gett_single(x, kKindZero, zero_ctas(x), dtype, s, pdl);
        pdl = true;
    }
    launch_gett_single(x, x.kind, desc_ctas(x), dtype, s, pdl);
    if (x.part) launch_gett_single(x, kKindReduce, reduce_ctas(x), dtype, s);
}

// A contraction planned once for fixed layouts (offset tables on the device,
// kernel choice, split-K and tensor-core workspaces) and run for any operand
// pointers with those layouts.
struct Prepared {
    GettDesc d;
    DevBuf tab, part, tcws;
    bool empty = false;
    int dtype = 0;
    Prepared(const Layout &A, const Layout &B, const Layout &C, int naxes, const int *axa,
             const int *axb, int dt, int precision, cudaStream_t s, int reduce_mode = kReduceAuto) {
        dtype = dt;
        memset(&d, 0, sizeof(d));
        GettView v = make_view(A, B, C, naxes, axa, axb);
        if (v.Mtot * v.Ntot == 0) {
            empty = true;
            return;
        }
        const TableLayout L = table_layout(v, gate_record_class(v, dt, precision, reduce_mode, 0));
        tab = DevBuf(L.entries * sizeof(int64_t), s);
        launch_build_tables(v, L, (int64_t *)tab.p, s);
        const int64_t *t = (const int64_t *)tab.p;
        fill_desc_tables(d, v, t + L.off[0], t + L.off[1], t + L.off[2]);
        choose_kernel(d, dt, precision, reduce_mode);
        if (is_tc()) {
            tcws = DevBuf(tc_workspace_bytes(d, packed_mode(d.kind)), s);
            tc_workspace_clear(d, packed_mode(d.kind), tcws.p, s);
        } else
            part = DevBuf(desc_part_bytes(d, dt), s);
        d.part = part.p;
    }
    bool is_tc() const { return is_packed_kind(d.kind); }
    // The first launch of the first run follows the kernel that built the
    // offset tables it reads in its prologue: it is launched in plain stream
    // order (see launch_pdl).
    bool tables_fresh = true;
    void run(rosnet_btensor A, rosnet_btensor B, rosnet_btensor C, cudaStream_t s, bool pack_b = true) {
        if (empty) return;
        GettDesc x = d;
        bind_operands(x, A->data, B->data, C->data, A->pstride, B->pstride, C->pstride);
        const bool pdl = !tables_fresh;
        tables_fresh = false;
        if (is_tc()) {
            GroupArgs ga;
            memset(&ga, 0, sizeof(ga));
            ga.ndesc = 1;
            ga.single = x;
            // after an operand swap the kernel's first operand is B
            const bool sw = x.flags & kFlagSwapped;
            launch_tc_problem(packed_mode(x.kind), x, ga, tcws.p, s, sw ? pack_b : true, sw ? true : pack_b, {},
                              pdl);
            return;
        }
        launch_sequence(x, dtype, s, pdl);
    }
};

void tensordot_into(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axa, const int *axb,
                    rosnet_btensor C, int precision, cudaStream_t s, int reduce_mode) {
    Prepared p(A->lay, B->lay, C->lay, naxes, axa, axb, A->dtype, precision, s, reduce_mode);
    p.run(A, B, C, s);
}

int check_reduce(const rosnet_opts *opts) {
    if (!opts) return kReduceAuto;
    const int f = opts->flags & (ROSNET_OPT_REDUCE_SEQUENTIAL | ROSNET_OPT_REDUCE_TREE |
                                 ROSNET_OPT_REDUCE_COMMUTATIVE);
    switch (f) {
        case 0: return kReduceAuto;
        case ROSNET_OPT_REDUCE_SEQUENTIAL: return kReduceSequential;
        case ROSNET_OPT_REDUCE_TREE: return kReduceTree;
        case ROSNET_OPT_REDUCE_COMMUTATIVE: return kReduceCommutative;
        default: RN_FAIL(ROSNET_ERR_INVALID_ARG, "at most one reduction flag");
    }
}


// The same contraction with caller-provided scratch instead of allocations:
// the offset tables and any split-K partials or packed operands are placed in
// `ws` (ws_bytes long, 256-byte aligned).  Returns the scratch bytes the
// problem needs; if that exceeds ws_bytes nothing is launched.  The kernel
// that builds the tables overwrites the previous call's in stream order (it
// starts only after all earlier work in the stream), and the launch after it
// waits for it to complete (pdl = false).
size_t tensordot_into_ws(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axa,
                         const int *axb, rosnet_btensor C, int precision, int reduce_mode, void *ws,
                         size_t ws_bytes, cudaStream_t s) {
    GettView v = make_view(A->lay, B->lay, C->lay, naxes, axa, axb);
    if (v.Mtot * v.Ntot == 0) return 0;
    GettDesc d;
    TableLayout L;
    size_t tab_bytes = 0;
    auto plan = [&](int red) {
        L = table_layout(v, gate_record_class(v, A->dtype, precision, red, 0));
        tab_bytes = (L.entries * sizeof(int64_t) + 255) & ~(size_t)255;
        const int64_t *t = (const int64_t *)ws;
        memset(&d, 0, sizeof(d));
        fill_desc_tables(d, v, t + L.off[0], t + L.off[1], t + L.off[2]);
        choose_kernel(d, A->dtype, precision, red);
        // the workspace for these operand addresses (no packed panels for
        // operands read in place)
        bind_operands(d, A->data, B->data, C->data, A->pstride, B->pstride, C->pstride);
        return tab_bytes + (is_packed_kind(d.kind) ? tc_workspace_bytes_bound(d, packed_mode(d.kind))
                                                   : desc_part_bytes(d, A->dtype));
    };
    size_t need = plan(reduce_mode);
    // an automatic split of the contracted range (or stream-K schedule) whose
    // partial sums do not fit runs unsplit instead (one CTA per output tile
    // over all pairs)
    if (need > ws_bytes && reduce_mode == kReduceAuto && (d.ksplit > 1 || (d.flags & kFlagStreamK)))
        need = plan(kReduceSequential);
    if (need > ws_bytes) return need;
    const bool tcp = is_packed_kind(d.kind);
    launch_build_tables(v, L, (int64_t *)ws, s);
    bind_operands(d, A->data, B->data, C->data, A->pstride, B->pstride, C->pstride);
    if (tcp) {
        GroupArgs ga;
        memset(&ga, 0, sizeof(ga));
        ga.ndesc = 1;
        ga.single = d;
        tc_workspace_clear(d, packed_mode(d.kind), (char *)ws + tab_bytes, s);
        launch_tc_problem(packed_mode(d.kind), d, ga, (char *)ws + tab_bytes, s, true, true, {}, false);
        return need;
    }
    d.part = desc_part_bytes(d, A->dtype) ? (char *)ws + tab_bytes : nullptr;
    launch_sequence(d, A->dtype, s, false);
    return need;
}

// Validate a tensordot request and return the shape/blocks of C.
void check_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axes_a,
                     const int *axes_b, int *axa, int *axb, int &rc, int64_t *shc, int64_t *blc) {
    if (!A || !B) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL operand");
    if (naxes < 0 || naxes > A->lay.rank || naxes > B->lay.rank)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad number of contracted axes");
    if (naxes > 0 && (!axes_a || !axes_b)) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL axes");
    if (A->dtype != B->dtype) RN_FAIL(ROSNET_ERR_DTYPE, "operands have different dtypes");
    bool ua[kMaxRank] = {false}, ub[kMaxRank] = {false};
    for (int i = 0; i < naxes; ++i) {
        int x = axes_a[i] < 0 ? axes_a[i] + A->lay.rank : axes_a[i];
        int y = axes_b[i] < 0 ? axes_b[i] + B->lay.rank : axes_b[i];
        if (x < 0 || x >= A->lay.rank || y < 0 || y >= B->lay.rank)
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "axis out of range");
        if (ua[x] || ub[y]) RN_FAIL(ROSNET_ERR_INVALID_ARG, "axis contracted twice");
        ua[x] = ub[y] = true;
        if (A->lay.shape[x] != B->lay.shape[y])
            RN_FAIL(ROSNET_ERR_SHAPE, "contracted axes have different extents");
        if (A->lay.block[x] != B->lay.block[y])
            RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "contracted axes have different block extents");
        axa[i] = x;
        axb[i] = y;
    }
    rc = 0;
    for (int i = 0; i < A->lay.rank; ++i)
        if (!ua[i]) {
            shc[rc] = A->lay.shape[i];
            blc[rc++] = A->lay.block[i];
        }
    for (int i = 0; i < B->lay.rank; ++i)
        if (!ub[i]) {
            if (rc >= kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "result rank > 64");
            shc[rc] = B->lay.shape[i];
            blc[rc++] = B->lay.block[i];
        }
}

int check_precision(const rosnet_opts *opts, int dtype) {
    if (!opts) return ROSNET_PREC_DEFAULT;
    for (int i = 0; i < 6; ++i)
        if (opts->reserved[i] != 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "reserved option fields must be 0");
    int p = opts->precision;
    if (p < ROSNET_PREC_DEFAULT || p > ROSNET_PREC_TF32X3) RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad precision");
    if (dtype == ROSNET_C128 && p != ROSNET_PREC_DEFAULT && p != ROSNET_PREC_FP64)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "complex128 supports the FP64 mode only");
    if (dtype == ROSNET_C64 && p == ROSNET_PREC_FP64)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "FP64 mode needs complex128 operands");
    return p;
}

}  // namespace rosnet

using namespace rosnet;

extern "C" rosnet_status rosnet_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes,
                                          const int *axes_a, const int *axes_b,
                                          const rosnet_opts *opts, void *stream,
                                          rosnet_btensor *out_C) {
    if (!out_C) return ROSNET_ERR_INVALID_ARG;
    *out_C = nullptr;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    int axa[kMaxRank], axb[kMaxRank], rc = 0;
    int64_t shc[kMaxRank], blc[kMaxRank];
    check_tensordot(A, B, naxes, axes_a, axes_b, axa, axb, rc, shc, blc);
    int prec = check_precision(opts, A->dtype);
    const int red = check_reduce(opts);
    rosnet_btensor C = new_tensor(rc, shc, blc, A->dtype, s);
    try {
        tensordot_into(A, B, naxes, axa, axb, C, prec, s, red);
    } catch (...) {
        free_tensor(C);
        throw;
    }
    *out_C = C;
    return ROSNET_OK;
    RN_API_END
}

// ---------------------------------------------------------------------------
// out-of-core: output chunks streamed to pinned host memory; A either on the
// device or, slice by slice, streamed in from host memory
// ---------------------------------------------------------------------------
namespace rosnet {
namespace {

// The chunk loop shared by both entry points.  A describes A's layout and
// dtype; with from_host set its data pointer is unused and chunk c's slice of
// A (a contiguous run of blocks in each plane, planes numel apart in the
// host array) is copied into one of two device buffers on an input stream,
// one chunk ahead of the computation; output chunk c goes out on a second
// side stream while chunk c + 1 is computed.
void ooc_run(rosnet_btensor A, bool from_host, const void *a_host, rosnet_btensor B, int naxes,
             const int *axes_a,
             const int *axes_b, int nsplit, int64_t first_chunk, int64_t nchunks, const rosnet_opts *opts,
             void *host_out, size_t host_bytes, cudaStream_t s) {
    if (!A || !B || nsplit < 0 || nsplit > A->lay.rank || first_chunk < 0 || nchunks < 0)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad operands or chunk range");
    int axa[kMaxRank], axb[kMaxRank], rc = 0;
    int64_t shc[kMaxRank], blc[kMaxRank];
    check_tensordot(A, B, naxes, axes_a, axes_b, axa, axb, rc, shc, blc);
    const int prec = check_precision(opts, A->dtype);
    // the split axes: A's leading axes, free and of block extent 1
    int64_t total_chunks = 1;
    for (int i = 0; i < nsplit; ++i) {
        for (int j = 0; j < naxes; ++j)
            if (axa[j] == i) RN_FAIL(ROSNET_ERR_INVALID_ARG, "a split axis of A is contracted");
        if (A->lay.block[i] != 1) RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "a split axis must be a grid axis");
        total_chunks *= A->lay.shape[i];
    }
    if (first_chunk + nchunks > total_chunks) RN_FAIL(ROSNET_ERR_INVALID_ARG, "chunk range beyond the output");
    // chunk tensors: the slice of A and the matching output piece
    int axa_s[kMaxRank];
    for (int j = 0; j < naxes; ++j) axa_s[j] = axa[j] - nsplit;
    Layout lc;
    lc.init(rc - nsplit, shc + nsplit, blc + nsplit);
    const size_t chunk_bytes = 2 * (size_t)lc.numel * A->elsize;
    const int64_t nslots = chunk_bytes ? (int64_t)(host_bytes / chunk_bytes) : 1;
    if (nchunks > 0 && (!host_out || nslots < 1))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "the host buffer cannot hold one output chunk");
    if (nchunks == 0) return;
    rosnet_btensor_s av;   // slice view of A (A's strides), re-pointed per chunk
    av.lay.rank = A->lay.rank - nsplit;
    av.lay.numel = 1;
    for (int a = 0; a < av.lay.rank; ++a) {
        av.lay.shape[a] = A->lay.shape[a + nsplit];
        av.lay.block[a] = A->lay.block[a + nsplit];
        av.lay.gstride[a] = A->lay.gstride[a + nsplit];
        av.lay.lstride[a] = A->lay.lstride[a + nsplit];
        av.lay.numel *= av.lay.shape[a];
    }
    av.dtype = A->dtype;
    av.elsize = A->elsize;
    av.pstride = from_host ? av.lay.numel : A->pstride;   // staged slices: planes back to back
    av.owned = false;
    const size_t slice_plane = (size_t)av.lay.numel * A->elsize;
    auto slice_offset = [&](int64_t c) {   // elements from A's start to chunk c's slice (one plane)
        int64_t rem = c, off = 0;
        for (int i = nsplit - 1; i >= 0; --i) {
            off += (rem % A->lay.shape[i]) * A->lay.gstride[i];
            rem /= A->lay.shape[i];
        }
        return off;
    };
    rosnet_btensor_s cv[2];
    DevBuf cbuf[2], abuf[2];
    cudaStream_t side = nullptr, ins = nullptr;
    cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr}, loaded[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        if (side) { cudaStreamSynchronize(side); cudaStreamDestroy(side); }
        if (ins) { cudaStreamSynchronize(ins); cudaStreamDestroy(ins); }
        for (int i = 0; i < 2; ++i) {
            if (computed[i]) cudaEventDestroy(computed[i]);
            if (copied[i]) cudaEventDestroy(copied[i]);
            if (loaded[i]) cudaEventDestroy(loaded[i]);
        }
    };
    try {
        RN_CHECK_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        if (from_host) RN_CHECK_CUDA(cudaStreamCreateWithFlags(&ins, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            RN_CHECK_CUDA(cudaEventCreateWithFlags(&computed[i], cudaEventDisableTiming));
            RN_CHECK_CUDA(cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming));
            RN_CHECK_CUDA(cudaEventCreateWithFlags(&loaded[i], cudaEventDisableTiming));
            cbuf[i] = DevBuf(chunk_bytes, s);
            if (from_host) abuf[i] = DevBuf(2 * slice_plane, s);
            cv[i].lay = lc;
            cv[i].dtype = A->dtype;
            cv[i].elsize = A->elsize;
            cv[i].data = cbuf[i].p;
            cv[i].pstride = lc.numel;
            cv[i].owned = false;
        }
        // the staging buffers come from the caller's stream: the input stream
        // starts after their allocation
        if (from_host) {
            RN_CHECK_CUDA(cudaEventRecord(loaded[0], s));
            RN_CHECK_CUDA(cudaStreamWaitEvent(ins, loaded[0], 0));
        }
        // chunk c's slice of A into buffer (c - first_chunk) % 2, once the
        // chunk that used that buffer before (c - 2) has been computed
        auto load = [&](int64_t c) {
            const int b = (int)((c - first_chunk) & 1);
            if (c - first_chunk >= 2) RN_CHECK_CUDA(cudaStreamWaitEvent(ins, computed[b], 0));
            if (slice_plane > 0) {
                const char *src = (const char *)a_host + (size_t)slice_offset(c) * A->elsize;
                const size_t host_plane = (size_t)A->lay.numel * A->elsize;
                RN_CHECK_CUDA(cudaMemcpyAsync(abuf[b].p, src, slice_plane, cudaMemcpyHostToDevice, ins));
                RN_CHECK_CUDA(cudaMemcpyAsync((char *)abuf[b].p + slice_plane, src + host_plane, slice_plane,
                                              cudaMemcpyHostToDevice, ins));
            }
            RN_CHECK_CUDA(cudaEventRecord(loaded[b], ins));
        };
        if (from_host) load(first_chunk);
        Prepared prep(av.lay, B->lay, lc, naxes, axa_s, axb, A->dtype, prec, s, check_reduce(opts));
        for (int64_t c = first_chunk; c < first_chunk + nchunks; ++c) {
            const int b = (int)((c - first_chunk) & 1);
            if (from_host) {
                if (c + 1 < first_chunk + nchunks) load(c + 1);   // the next slice streams in meanwhile
                RN_CHECK_CUDA(cudaStreamWaitEvent(s, loaded[b], 0));
                av.data = abuf[b].p;
            } else {
                av.data = (char *)A->data + slice_offset(c) * A->elsize;
            }
            if (c - first_chunk >= 2) RN_CHECK_CUDA(cudaStreamWaitEvent(s, copied[b], 0));
            prep.run(&av, B, &cv[b], s, c == first_chunk);   // B is packed once
            RN_CHECK_CUDA(cudaEventRecord(computed[b], s));
            RN_CHECK_CUDA(cudaStreamWaitEvent(side, computed[b], 0));
            char *dst = (char *)host_out + ((c - first_chunk) % nslots) * chunk_bytes;
            RN_CHECK_CUDA(cudaMemcpyAsync(dst, cv[b].data, chunk_bytes, cudaMemcpyDeviceToHost, side));
            RN_CHECK_CUDA(cudaEventRecord(copied[b], side));
        }
        // the caller's stream waits for the last copies (and the staging
        // buffers are released on it after the last computation)
        for (int i = 0; i < 2; ++i) RN_CHECK_CUDA(cudaStreamWaitEvent(s, copied[i], 0));
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();   // synchronises the side streams (the copies are complete on return)
}

}  // namespace
}  // namespace rosnet

extern "C" rosnet_status rosnet_tensordot_ooc(rosnet_btensor A, rosnet_btensor B, int naxes,
                                              const int *axes_a, const int *axes_b, int nsplit,
                                              int64_t first_chunk, int64_t nchunks,
                                              const rosnet_opts *opts, void *host_out,
                                              size_t host_bytes, void *stream) {
    RN_API_BEGIN
    ooc_run(A, false, nullptr, B, naxes, axes_a, axes_b, nsplit, first_chunk, nchunks, opts, host_out, host_bytes,
            (cudaStream_t)stream);
    return ROSNET_OK;
    RN_API_END
}

extern "C" rosnet_status rosnet_tensordot_ooc_host(int rank_a, const int64_t *shape_a, const int64_t *block_a,
                                                   const void *a_host, rosnet_btensor B, int naxes,
                                                   const int *axes_a, const int *axes_b, int nsplit,
                                                   int64_t first_chunk, int64_t nchunks,
                                                   const rosnet_opts *opts, void *host_out,
                                                   size_t host_bytes, void *stream) {
    RN_API_BEGIN
    if (!B || rank_a < 0 || rank_a > kMaxRank || (rank_a > 0 && !shape_a))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad operand description");
    rosnet_btensor_s a;   // A's layout and dtype only: its data stay in host memory
    a.lay.init(rank_a, shape_a, block_a);
    a.dtype = B->dtype;
    a.elsize = B->elsize;
    a.pstride = a.lay.numel;
    a.owned = false;
    if (!a_host && a.lay.numel > 0 && nchunks > 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no host array for A");
    ooc_run(&a, true, a_host, B, naxes, axes_a, axes_b, nsplit, first_chunk, nchunks, opts, host_out, host_bytes,
            (cudaStream_t)stream);
    return ROSNET_OK;
    RN_API_END
}

extern "C" rosnet_status rosnet_tune_export(char *buf, size_t cap, size_t *len) {
    using namespace rosnet;
    if (!len) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    std::string t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &e : g_tune) {
            const TuneKey &k = e.first;
            const TuneChoice &c = e.second;
            t += std::to_string(k.dtype) + " " + std::to_string(k.flags) + " " + std::to_string(k.M) + " " +
                 std::to_string(k.N) + " " + std::to_string(k.K) + " " + std::to_string(c.kind) + " " +
                 std::to_string(c.ksplit) + " " + std::to_string((c.flags & kFlagStreamK) ? 1 : 0) + "\n";
        }
    }
    *len = t.size() + 1;
    if (buf && cap >= t.size() + 1) memcpy(buf, t.c_str(), t.size() + 1);
    return ROSNET_OK;
    RN_API_END
}

extern "C" rosnet_status rosnet_tune_import(const char *text) {
    using namespace rosnet;
    if (!text) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    std::vector<std::pair<TuneKey, TuneChoice>> add;
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
        std::istringstream ls(line);
        long long v[8] = {0};
        for (int i = 0; i < 7; ++i)
            if (!(ls >> v[i])) RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed tuning line: " + line);
        if (ls >> v[7]) {   // optional: the packed FP32 GEMM's stream-K schedule (0 / 1)
            if (v[7] != 0 && (v[7] != 1 || v[5] != kKindPackF32))
                RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad schedule field: " + line);
        } else if (!ls.eof()) {
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed tuning line: " + line);
        }
        std::string rest;
        ls.clear();
        if (ls >> rest) RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed tuning line: " + line);
        if (v[0] != ROSNET_C64 && v[0] != ROSNET_C128) RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad dtype: " + line);
        if (v[1] < 0 || v[1] > 0x7fffffffLL)
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad tuning line: " + line);
        TuneChoice c;
        if (!tune_geometry((int)v[0], (int)v[5], v[2], v[3], v[4], v[6], &c))
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "choice impossible for this shape: " + line);
        c.flags = v[7] ? kFlagStreamK : 0;
        add.push_back({TuneKey{(int)v[0], (int)v[1], v[2], v[3], v[4]}, c});
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : add) g_tune[e.first] = e.second;
    return ROSNET_OK;
    RN_API_END
}
