// Allocator, block layouts, tensor handles and layout-changing copies.
//
// Block tensors (Sec. II-C): a tensor is cut into a uniform grid of blocks;
// on the device the blocks are stored one after another (row-major over the
// grid coordinates), each block row-major inside, with all real parts first
// and all imaginary parts after them (planar complex).
#include <cuda_runtime.h>

#include <atomic>

#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

namespace rosnet {

std::atomic<int64_t> g_launches{0};

int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];   // 0 = not yet queried
    int dev = 0;
    RN_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "device index out of range");
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        RN_CHECK_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        if (n <= 0) RN_FAIL(ROSNET_ERR_CUDA, "device reports no multiprocessors");
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

static thread_local std::string t_last_error;
void set_last_error(const std::string &s) { t_last_error = s; }
const char *last_error_cstr() { return t_last_error.c_str(); }

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
static void *(*g_alloc)(size_t, void *, void *) = nullptr;
static void (*g_free)(void *, void *, void *) = nullptr;
static void *g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_live_allocs{0};   // blocks handed out and not yet freed
static std::atomic<int64_t> g_alloc_requests{0};   // blocks handed out in total

// The built-in allocator draws on the device's default stream-ordered pool;
// freed blocks stay in the pool across synchronisations (release threshold
// raised once per device, for this process) so that steady-state calls do
// not map and unmap memory.
static void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, (void *)s, g_alloc_ctx);
        if (!p) RN_FAIL(ROSNET_ERR_ALLOC, "injected allocator returned NULL for " +
                                              std::to_string(bytes) + " bytes");
        ++g_live_allocs;
        ++g_alloc_requests;
        return p;
    }
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        RN_FAIL(ROSNET_ERR_ALLOC, "cudaMallocAsync(" + std::to_string(bytes) +
                                      "): " + cudaGetErrorString(e));
    }
    ++g_live_allocs;
    ++g_alloc_requests;
    return p;
}

void dev_free(void *p, cudaStream_t s) {
    if (!p) return;
    --g_live_allocs;
    if (g_free) {
        g_free(p, (void *)s, g_alloc_ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------
// layouts
// ---------------------------------------------------------------------------
void Layout::init(int r, const int64_t *sh, const int64_t *bl) {
    if (r < 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "negative rank");
    if (r > kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "rank " + std::to_string(r) + " > 64");
    if (r > 0 && !sh) RN_FAIL(ROSNET_ERR_INVALID_ARG, "shape is NULL");
    rank = r;
    numel = 1;
    for (int i = 0; i < r; ++i) {
        if (sh[i] < 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "negative extent");
        int64_t b = bl ? bl[i] : (sh[i] > 0 ? sh[i] : 1);
        if (b < 1) RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "block extent < 1");
        if (sh[i] % b != 0)
            RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "block extent " + std::to_string(b) +
                                                   " does not divide extent " +
                                                   std::to_string(sh[i]) + " of axis " +
                                                   std::to_string(i));
        shape[i] = sh[i];
        block[i] = b;
        if (sh[i] > 0 && numel > kMaxNumel / sh[i])
            RN_FAIL(ROSNET_ERR_SHAPE, "tensor too large (more than 2^58 elements)");
        numel *= sh[i];
    }
    int64_t bs = 1;
    for (int i = r - 1; i >= 0; --i) {
        lstride[i] = bs;
        bs *= block[i];
    }
    int64_t g = bs;
    for (int i = r - 1; i >= 0; --i) {
        gstride[i] = g;
        g *= shape[i] / block[i];
    }
}

// ---------------------------------------------------------------------------
// strided copies between layouts
// ---------------------------------------------------------------------------
// Modes of a copy, innermost last: element e (enumerated row-major over the
// modes) is read at sum d_j*ss_j and written at sum d_j*ds_j.
struct CopyModes {
    int n;
    int pow2;                 // all extents are powers of two
    int64_t ext[kMaxModes];
    int64_t ss[kMaxModes];
    int64_t ds[kMaxModes];
};

static void push_mode(CopyModes &cm, int64_t ext, int64_t ss, int64_t ds) {
    if (ext == 1) return;
    if (cm.n > 0) {  // fuse with the previous (outer) mode when contiguous in both
        int j = cm.n - 1;
        if (cm.ss[j] == ss * ext && cm.ds[j] == ds * ext) {
            cm.ext[j] *= ext;
            cm.ss[j] = ss;
            cm.ds[j] = ds;
            return;
        }
    }
    if (cm.n >= kMaxModes) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "too many modes");
    cm.ext[cm.n] = ext;
    cm.ss[cm.n] = ss;
    cm.ds[cm.n] = ds;
    cm.n++;
}

static void finish_modes(CopyModes &cm) {
    cm.pow2 = 1;
    for (int i = 0; i < cm.n; ++i)
        if (cm.ext[i] & (cm.ext[i] - 1)) cm.pow2 = 0;
}

// The digits of one logical axis of extent s under the two block extents
// b_src and b_dst (one must divide the other): modes from outer to inner with
// their strides in both layouts.
static void axis_modes(CopyModes &cm, int64_t s, int64_t b1, int64_t g1, int64_t l1,
                       int64_t b2, int64_t g2, int64_t l2) {
    int64_t lo = b1 < b2 ? b1 : b2, hi = b1 < b2 ? b2 : b1;
    if (hi % lo) RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "block extents are not nested");
    // levels (units): hi, lo, 1 ; a digit with unit u has stride
    // (u >= b ? g * (u / b) : l * u) in a layout with block b
    auto st = [](int64_t u, int64_t b, int64_t g, int64_t l) { return u >= b ? g * (u / b) : l * u; };
    push_mode(cm, s / hi, st(hi, b1, g1, l1), st(hi, b2, g2, l2));
    push_mode(cm, hi / lo, st(lo, b1, g1, l1), st(lo, b2, g2, l2));
    push_mode(cm, lo, st(1, b1, g1, l1), st(1, b2, g2, l2));
}

template <typename T, int MODE>  // MODE 0: interleaved->planar, 1: planar->interleaved, 2: planar->planar
__global__ void __launch_bounds__(256) copy_modes_kernel(CopyModes cm, int64_t total, int64_t first,
                                                         const T *__restrict__ src, int64_t src_plane,
                                                         T *__restrict__ dst, int64_t dst_plane) {
    // elements [first, first + total) of the enumeration; the source of MODE 0
    // holds only that range (it starts at element `first`)
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; e < total; e += stride) {
        int64_t r = e + first, so = 0, dof = 0;
        if (cm.pow2) {
            for (int j = cm.n - 1; j >= 0; --j) {
                int64_t x = cm.ext[j];
                int64_t d = r & (x - 1);
                r >>= __popcll(x - 1);
                so += d * cm.ss[j];
                dof += d * cm.ds[j];
            }
        } else {
            for (int j = cm.n - 1; j >= 0; --j) {
                int64_t d = r % cm.ext[j];
                r /= cm.ext[j];
                so += d * cm.ss[j];
                dof += d * cm.ds[j];
            }
        }
        T re, im;
        if (MODE == 0) {
            re = src[2 * (so - first)];
            im = src[2 * (so - first) + 1];
        } else {
            re = src[so];
            im = src[so + src_plane];
        }
        if (MODE == 1) {
            dst[2 * dof] = re;
            dst[2 * dof + 1] = im;
        } else {
            dst[dof] = re;
            dst[dof + dst_plane] = im;
        }
    }
}

static int copy_grid(int64_t total) {
    int64_t b = (total + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int MODE>
static void launch_copy(const CopyModes &cm, int64_t total, int dtype, const void *src,
                        int64_t src_plane, void *dst, int64_t dst_plane, cudaStream_t s,
                        int64_t first = 0) {
    if (total == 0) return;
    if (dtype == ROSNET_C64)
        copy_modes_kernel<float, MODE><<<copy_grid(total), 256, 0, s>>>(
            cm, total, first, (const float *)src, src_plane, (float *)dst, dst_plane);
    else
        copy_modes_kernel<double, MODE><<<copy_grid(total), 256, 0, s>>>(
            cm, total, first, (const double *)src, src_plane, (double *)dst, dst_plane);
    g_launches++;
    RN_CHECK_CUDA(cudaGetLastError());
}

// Modes of "dense row-major" <-> "block-major" for one layout.  Elements are
// enumerated in row-major order of the dense tensor.
static CopyModes dense_block_modes(const Layout &lay) {
    CopyModes cm{};
    int64_t rs = 1;
    int64_t rstride[kMaxRank];
    for (int i = lay.rank - 1; i >= 0; --i) {
        rstride[i] = rs;
        rs *= lay.shape[i];
    }
    for (int i = 0; i < lay.rank; ++i) {
        int64_t s = lay.shape[i], b = lay.block[i];
        // dense row-major: block "s" (one block); block-major: block b
        axis_modes(cm, s, s, 0, rstride[i], b, lay.gstride[i], lay.lstride[i]);
    }
    finish_modes(cm);
    return cm;
}

void launch_pack(const Layout &lay, int dtype, const void *dense, void *planar, int64_t pstride,
                 int64_t start, int64_t count, cudaStream_t s) {
    if (lay.numel == 0 || count == 0) return;
    CopyModes cm = dense_block_modes(lay);
    launch_copy<0>(cm, count, dtype, dense, 0, planar, pstride, s, start);
}

void launch_unpack(const Layout &lay, int dtype, const void *planar, int64_t pstride, void *dense,
                   cudaStream_t s) {
    if (lay.numel == 0) return;
    CopyModes cm = dense_block_modes(lay);
    // enumerate in dense order: ss = block-major (source), ds = dense (dest)
    for (int j = 0; j < cm.n; ++j) {
        int64_t t = cm.ss[j];
        cm.ss[j] = cm.ds[j];
        cm.ds[j] = t;
    }
    launch_copy<1>(cm, lay.numel, dtype, planar, pstride, dense, 0, s);
}

void launch_relayout(const Layout &src, const Layout &dst, const int *perm, int dtype,
                     const void *sp, int64_t spstride, void *dp, int64_t dpstride, cudaStream_t s) {
    if (dst.numel == 0) return;
    // enumerate in destination axis order
    CopyModes cm{};
    for (int i = 0; i < dst.rank; ++i) {
        int a = perm[i];
        if (src.shape[a] != dst.shape[i]) RN_FAIL(ROSNET_ERR_SHAPE, "relayout shape mismatch");
        axis_modes(cm, dst.shape[i], src.block[a], src.gstride[a], src.lstride[a], dst.block[i],
                   dst.gstride[i], dst.lstride[i]);
    }
    finish_modes(cm);
    launch_copy<2>(cm, dst.numel, dtype, sp, spstride, dp, dpstride, s);
}

// Sum of |x|^2 over a tensor in FP64: every thread of a fixed grid adds the
// elements i = tid, tid + grid, ... (logical row-major index, offsets from
// the layout, so views work), the block's threads are summed in a fixed
// tree, and one block adds the per-block partials in block order: a fixed
// order for a given grid, so the result is reproducible.
template <typename T>
__global__ void __launch_bounds__(256) norm2_partial_kernel(Layout lay, const T *__restrict__ re, int64_t pstride,
                                                             double *__restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < lay.numel; i += (int64_t)gridDim.x * 256) {
        int64_t r = i, off = 0;
        for (int a = lay.rank - 1; a >= 0; --a) {
            const int64_t x = r % lay.shape[a];
            r /= lay.shape[a];
            off += (x / lay.block[a]) * lay.gstride[a] + (x % lay.block[a]) * lay.lstride[a];
        }
        const double xr = (double)re[off], xi = (double)re[off + pstride];
        acc = fma(xr, xr, acc);
        acc = fma(xi, xi, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void norm2_final_kernel(const double *__restrict__ part, int nparts, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int j = 0; j < nparts; ++j) s += part[j];
        *out = s;
    }
}

// out[i] = sum_j in_j[i] in FP64, j in order (deterministic); inputs complex64
// or complex128 planar with plane strides ps[j], output complex128 planar.
template <typename T>
__global__ void __launch_bounds__(256) sum_fp64_kernel(const T *const *__restrict__ in,
                                                       const int64_t *__restrict__ ps, int n,
                                                       int64_t numel, double *__restrict__ out,
                                                       int64_t ops) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < numel;
         i += (int64_t)gridDim.x * blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            sr += (double)in[j][i];
            si += (double)in[j][i + ps[j]];
        }
        out[i] = sr;
        out[i + ops] = si;
    }
}

// ---------------------------------------------------------------------------
// tensors
// ---------------------------------------------------------------------------
rosnet_btensor new_tensor(int rank, const int64_t *shape, const int64_t *block, int dtype,
                          cudaStream_t s) {
    if (dtype != ROSNET_C64 && dtype != ROSNET_C128) RN_FAIL(ROSNET_ERR_DTYPE, "unknown dtype");
    rosnet_btensor t = new rosnet_btensor_s();
    try {
        t->lay.init(rank, shape, block);
        t->dtype = dtype;
        t->elsize = dtype == ROSNET_C64 ? 4 : 8;
        t->stream = s;
        t->data = dev_alloc(2 * t->lay.numel * t->elsize, s);
        t->pstride = t->lay.numel;
    } catch (...) {
        delete t;
        throw;
    }
    return t;
}

void free_tensor(rosnet_btensor t) {
    if (!t) return;
    if (t->owned && t->data) dev_free(t->data, t->stream);
    delete t;
}

}  // namespace rosnet

using namespace rosnet;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

rosnet_status rosnet_alloc_stats(int64_t *requests, int64_t *live) {
    if (requests) *requests = g_alloc_requests.load();
    if (live) *live = g_live_allocs.load();
    return ROSNET_OK;
}

rosnet_status rosnet_set_allocator(void *(*alloc)(size_t, void *, void *),
                                   void (*freef)(void *, void *, void *), void *ctx) {
    if ((alloc == nullptr) != (freef == nullptr)) return ROSNET_ERR_INVALID_ARG;
    // a block must be freed by the allocator that made it
    if (g_live_allocs.load() != 0 && (alloc != g_alloc || freef != g_free || ctx != g_alloc_ctx))
        return ROSNET_ERR_INVALID_ARG;
    g_alloc = alloc;
    g_free = freef;
    g_alloc_ctx = ctx;
    return ROSNET_OK;
}

rosnet_status rosnet_btensor_create(int rank, const int64_t *shape, const int64_t *block_shape,
                                    rosnet_dtype dtype, void *stream, rosnet_btensor *out) {
    if (!out) return ROSNET_ERR_INVALID_ARG;
    *out = nullptr;
    RN_API_BEGIN
    *out = new_tensor(rank, shape, block_shape, (int)dtype, (cudaStream_t)stream);
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_destroy(rosnet_btensor t) {
    RN_API_BEGIN
    free_tensor(t);
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_upload(rosnet_btensor t, const void *host, void *stream) {
    if (!t || (!host && t->lay.numel > 0)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = 2 * t->lay.numel * t->elsize;
    if (bytes == 0) return ROSNET_OK;
    DevBuf stage(bytes, s);
    RN_CHECK_CUDA(cudaMemcpyAsync(stage.p, host, bytes, cudaMemcpyHostToDevice, s));
    launch_pack(t->lay, t->dtype, stage.p, t->data, t->pstride, 0, t->lay.numel, s);
    if (t->owned) t->stream = s;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_upload_range(rosnet_btensor t, const void *host, int64_t start,
                                          int64_t count, void *stream) {
    if (!t || start < 0 || count < 0 || start > t->lay.numel || count > t->lay.numel - start ||
        (!host && count > 0))
        return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = 2 * (size_t)count * t->elsize;
    if (bytes == 0) return ROSNET_OK;
    DevBuf stage(bytes, s);
    RN_CHECK_CUDA(cudaMemcpyAsync(stage.p, host, bytes, cudaMemcpyHostToDevice, s));
    launch_pack(t->lay, t->dtype, stage.p, t->data, t->pstride, start, count, s);
    if (t->owned) t->stream = s;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_norm2(rosnet_btensor t, void *stream, double *out) {
    if (!t || !out) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const int nparts = num_sms() * 4;
    DevBuf buf((size_t)(nparts + 1) * sizeof(double), s);
    double *part = (double *)buf.p, *res = part + nparts;
    if (t->lay.numel == 0) {
        *out = 0.0;
        return ROSNET_OK;
    }
    if (t->dtype == ROSNET_C64)
        rosnet::norm2_partial_kernel<float><<<nparts, 256, 0, s>>>(t->lay, (const float *)t->data, t->pstride, part);
    else
        rosnet::norm2_partial_kernel<double><<<nparts, 256, 0, s>>>(t->lay, (const double *)t->data, t->pstride, part);
    rosnet::norm2_final_kernel<<<1, 32, 0, s>>>(part, nparts, res);
    g_launches += 2;
    RN_CHECK_CUDA(cudaGetLastError());
    double h = 0.0;
    RN_CHECK_CUDA(cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, s));
    RN_CHECK_CUDA(cudaStreamSynchronize(s));
    *out = h;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_sum(int32_t n, const rosnet_btensor *ts, void *stream, rosnet_btensor *out) {
    if (!out) return ROSNET_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !ts) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const rosnet_btensor t0 = ts[0];
    if (!t0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL tensor");
    for (int j = 0; j < n; ++j) {
        const rosnet_btensor t = ts[j];
        if (!t) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL tensor");
        if (t->dtype != t0->dtype) RN_FAIL(ROSNET_ERR_DTYPE, "summands differ in dtype");
        bool same = t->lay.rank == t0->lay.rank;
        for (int a = 0; same && a < t->lay.rank; ++a)
            same = t->lay.shape[a] == t0->lay.shape[a] && t->lay.block[a] == t0->lay.block[a] &&
                   t->lay.gstride[a] == t0->lay.gstride[a] && t->lay.lstride[a] == t0->lay.lstride[a];
        if (!same) RN_FAIL(ROSNET_ERR_SHAPE, "summands differ in shape, blocks or strides");
    }
    Layout canon;
    canon.init(t0->lay.rank, t0->lay.shape, t0->lay.block);
    for (int a = 0; a < canon.rank; ++a)
        if (canon.gstride[a] != t0->lay.gstride[a] || canon.lstride[a] != t0->lay.lstride[a])
            RN_FAIL(ROSNET_ERR_UNSUPPORTED, "summands must be dense block-major tensors");
    rosnet_btensor C = new_tensor(canon.rank, canon.shape, canon.block, ROSNET_C128, s);
    try {
        std::vector<const void *> hp(n);
        std::vector<int64_t> hs(n);
        for (int j = 0; j < n; ++j) {
            hp[j] = ts[j]->data;
            hs[j] = ts[j]->pstride;
        }
        DevBuf dp(n * sizeof(void *), s), dps(n * sizeof(int64_t), s);
        RN_CHECK_CUDA(cudaMemcpyAsync(dp.p, hp.data(), n * sizeof(void *), cudaMemcpyHostToDevice, s));
        RN_CHECK_CUDA(cudaMemcpyAsync(dps.p, hs.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        const int64_t numel = canon.numel;
        const int grid = (int)std::min<int64_t>(std::max<int64_t>((numel + 255) / 256, 1),
                                                        (int64_t)num_sms() * 8);
        if (numel > 0) {
            if (t0->dtype == ROSNET_C64)
                sum_fp64_kernel<float><<<grid, 256, 0, s>>>((const float *const *)dp.p, (const int64_t *)dps.p,
                                                            n, numel, (double *)C->data, C->pstride);
            else
                sum_fp64_kernel<double><<<grid, 256, 0, s>>>((const double *const *)dp.p,
                                                             (const int64_t *)dps.p, n, numel,
                                                             (double *)C->data, C->pstride);
            g_launches++;
            RN_CHECK_CUDA(cudaGetLastError());
        }
    } catch (...) {
        free_tensor(C);
        throw;
    }
    *out = C;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_fix(rosnet_btensor t, int nfix, const int *axes, const int64_t *values,
                                 rosnet_btensor *view) {
    if (!view) return ROSNET_ERR_INVALID_ARG;
    *view = nullptr;
    if (!t || nfix < 0 || nfix > t->lay.rank || (nfix > 0 && (!axes || !values))) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    bool fixed[kMaxRank] = {false};
    int64_t off = 0;
    for (int j = 0; j < nfix; ++j) {
        const int a = axes[j];
        if (a < 0 || a >= t->lay.rank || fixed[a]) RN_FAIL(ROSNET_ERR_INVALID_ARG, "bad or repeated axis");
        if (values[j] < 0 || values[j] >= t->lay.shape[a]) RN_FAIL(ROSNET_ERR_INVALID_ARG, "index out of range");
        fixed[a] = true;
        const int64_t b = t->lay.block[a];
        off += (values[j] / b) * t->lay.gstride[a] + (values[j] % b) * t->lay.lstride[a];
    }
    rosnet_btensor v = new rosnet_btensor_s();
    Layout &L = v->lay;
    L.rank = 0;
    L.numel = 1;
    for (int a = 0; a < t->lay.rank; ++a) {
        if (fixed[a]) continue;
        L.shape[L.rank] = t->lay.shape[a];
        L.block[L.rank] = t->lay.block[a];
        L.gstride[L.rank] = t->lay.gstride[a];
        L.lstride[L.rank] = t->lay.lstride[a];
        L.numel *= t->lay.shape[a];
        L.rank++;
    }
    v->dtype = t->dtype;
    v->elsize = t->elsize;
    v->data = (char *)t->data + off * t->elsize;
    v->pstride = t->pstride;
    v->stream = t->stream;
    v->owned = false;
    *view = v;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_block(rosnet_btensor t, const int64_t *grid_coords, rosnet_btensor *view) {
    if (!view) return ROSNET_ERR_INVALID_ARG;
    *view = nullptr;
    if (!t || (t->lay.rank > 0 && !grid_coords)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    int64_t off = 0;
    for (int i = 0; i < t->lay.rank; ++i) {
        const int64_t g = t->lay.shape[i] / t->lay.block[i];
        if (grid_coords[i] < 0 || grid_coords[i] >= g) RN_FAIL(ROSNET_ERR_INVALID_ARG, "block coordinate out of range");
        off += grid_coords[i] * t->lay.gstride[i];
    }
    rosnet_btensor v = new rosnet_btensor_s();
    try {
        v->lay.init(t->lay.rank, t->lay.block, t->lay.block);
    } catch (...) {
        delete v;
        throw;
    }
    v->dtype = t->dtype;
    v->elsize = t->elsize;
    v->data = (char *)t->data + off * t->elsize;
    v->pstride = t->pstride;
    v->stream = t->stream;
    v->owned = false;
    *view = v;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_slice(rosnet_btensor t, int nfix, const int64_t *values,
                                   rosnet_btensor *view) {
    if (!view) return ROSNET_ERR_INVALID_ARG;
    *view = nullptr;
    if (!t || nfix < 0 || nfix > t->lay.rank || (nfix > 0 && !values)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    int64_t off = 0;
    for (int i = 0; i < nfix; ++i) {
        if (values[i] < 0 || values[i] >= t->lay.shape[i])
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "slice index out of range");
        if (t->lay.block[i] != 1)
            RN_FAIL(ROSNET_ERR_BLOCK_MISMATCH, "a sliced axis must have block extent 1 (a grid axis)");
        off += values[i] * t->lay.gstride[i];
    }
    rosnet_btensor v = new rosnet_btensor_s();
    Layout &L = v->lay;
    L.rank = t->lay.rank - nfix;
    L.numel = 1;
    for (int a = 0; a < L.rank; ++a) {
        L.shape[a] = t->lay.shape[a + nfix];
        L.block[a] = t->lay.block[a + nfix];
        L.gstride[a] = t->lay.gstride[a + nfix];
        L.lstride[a] = t->lay.lstride[a + nfix];
        L.numel *= L.shape[a];
    }
    v->dtype = t->dtype;
    v->elsize = t->elsize;
    v->data = (char *)t->data + off * t->elsize;
    v->pstride = t->pstride;
    v->stream = t->stream;
    v->owned = false;
    *view = v;
    return ROSNET_OK;
    RN_API_END
}

static void download_enqueue(rosnet_btensor t, void *host, cudaStream_t s) {
    size_t bytes = 2 * t->lay.numel * t->elsize;
    if (bytes == 0) return;
    DevBuf stage(bytes, s);   // freed stream-ordered, after the copy
    launch_unpack(t->lay, t->dtype, t->data, t->pstride, stage.p, s);
    RN_CHECK_CUDA(cudaMemcpyAsync(host, stage.p, bytes, cudaMemcpyDeviceToHost, s));
}

rosnet_status rosnet_btensor_download(rosnet_btensor t, void *host, void *stream) {
    if (!t || (!host && t->lay.numel > 0)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    download_enqueue(t, host, s);
    RN_CHECK_CUDA(cudaStreamSynchronize(s));
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_download_async(rosnet_btensor t, void *host, void *stream) {
    if (!t || (!host && t->lay.numel > 0)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    download_enqueue(t, host, (cudaStream_t)stream);
    return ROSNET_OK;
    RN_API_END
}

static void check_raw(rosnet_btensor t) {
    if (!t->owned || t->pstride != t->lay.numel)
        RN_FAIL(ROSNET_ERR_UNSUPPORTED, "raw copies need a tensor that owns its storage (not a view)");
}

rosnet_status rosnet_btensor_upload_raw(rosnet_btensor t, const void *host, void *stream) {
    if (!t || (!host && t->lay.numel > 0)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    check_raw(t);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = 2 * (size_t)t->lay.numel * t->elsize;
    if (bytes) RN_CHECK_CUDA(cudaMemcpyAsync(t->data, host, bytes, cudaMemcpyDefault, s));
    t->stream = s;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_download_raw(rosnet_btensor t, void *host, void *stream) {
    if (!t || (!host && t->lay.numel > 0)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    check_raw(t);
    const size_t bytes = 2 * (size_t)t->lay.numel * t->elsize;
    if (bytes) RN_CHECK_CUDA(cudaMemcpyAsync(host, t->data, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_btensor_info(rosnet_btensor t, int *rank, int64_t *shape, int64_t *block_shape,
                                  rosnet_dtype *dtype) {
    if (!t || !rank) return ROSNET_ERR_INVALID_ARG;
    *rank = t->lay.rank;
    for (int i = 0; i < t->lay.rank; ++i) {
        if (shape) shape[i] = t->lay.shape[i];
        if (block_shape) block_shape[i] = t->lay.block[i];
    }
    if (dtype) *dtype = (rosnet_dtype)t->dtype;
    return ROSNET_OK;
}

rosnet_status rosnet_btensor_planes(rosnet_btensor t, void **re, void **im) {
    if (!t) return ROSNET_ERR_INVALID_ARG;
    if (re) *re = t->re();
    if (im) *im = t->im();
    return ROSNET_OK;
}

rosnet_status rosnet_sync(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        rosnet::set_last_error(cudaGetErrorString(e));
        return ROSNET_ERR_CUDA;
    }
    RN_API_BEGIN
    if (rosnet::take_device_status() != 0) {
        rosnet::set_last_error("a kernel gave up a bounded wait");
        return ROSNET_ERR_TIMEOUT;
    }
    return ROSNET_OK;
    RN_API_END
}

const char *rosnet_status_string(rosnet_status s) {
    switch (s) {
        case ROSNET_OK: return "ok";
        case ROSNET_ERR_INVALID_ARG: return "invalid argument";
        case ROSNET_ERR_SHAPE: return "shape mismatch";
        case ROSNET_ERR_BLOCK_MISMATCH: return "block shape mismatch";
        case ROSNET_ERR_DTYPE: return "dtype mismatch";
        case ROSNET_ERR_ALLOC: return "allocation failed";
        case ROSNET_ERR_RANK_LIMIT: return "rank limit exceeded";
        case ROSNET_ERR_CUDA: return "CUDA error";
        case ROSNET_ERR_TIMEOUT: return "device wait timed out";
        case ROSNET_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int64_t rosnet_kernel_launches(void) { return rosnet::g_launches.load(); }

const char *rosnet_last_error(void) { return rosnet::last_error_cstr(); }

}  // extern "C"
