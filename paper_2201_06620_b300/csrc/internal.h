// Internal declarations of librosnet (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/rosnet.h"

namespace rosnet {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
    rosnet_status code;
    std::string what;
};

#define RN_CHECK_CUDA(expr)                                             \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) throw ::rosnet::Error{ROSNET_ERR_CUDA,   \
                                   std::string(#expr) + ": " +         \
                                   cudaGetErrorString(_e)};             \
    } while (0)

#define RN_FAIL(code, msg) throw ::rosnet::Error{(code), (msg)}

void set_last_error(const std::string &s);
const char *last_error_cstr();

#define RN_API_BEGIN try {
#define RN_API_END                                   \
    }                                                \
    catch (const rosnet::Error &e) {                 \
        rosnet::set_last_error(e.what);              \
        return e.code;                               \
    }                                                \
    catch (const std::bad_alloc &) {                 \
        rosnet::set_last_error("host out of memory"); \
        return ROSNET_ERR_ALLOC;                     \
    }                                                \
    catch (...) {                                    \
        rosnet::set_last_error("unknown error");     \
        return ROSNET_ERR_INVALID_ARG;               \
    }


extern std::atomic<int64_t> g_launches;

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// queried once per device).  Grid sizes and the split heuristics scale with it.
int num_sms();

// A kernel's function attributes (its dynamic shared-memory limit) are set
// per device: `done` holds one bit per device index on which they are set.
// Returns the current device's bit, 0 if it is not set yet (then set the
// attributes and or the bit into `done`).  Setting them twice is harmless.
inline uint64_t attrs_set(const std::atomic<uint64_t> &done, uint64_t *bit) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 63;
    *bit = uint64_t(1) << dev;
    return done.load(std::memory_order_acquire) & *bit;
}

// Read and clear the device status word written by kernels whose bounded
// waits gave up (0 = none).
int32_t take_device_status();

// ---------------------------------------------------------------------------
// memory: the injected (or built-in stream-ordered) allocator
// ---------------------------------------------------------------------------
void *dev_alloc(size_t bytes, cudaStream_t s);      // throws ALLOC on failure
void dev_free(void *p, cudaStream_t s);

// RAII buffer in stream order
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t st) : bytes(n), s(st) { p = n ? dev_alloc(n, st) : nullptr; }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { reset(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; }
        return *this;
    }
    void reset() { if (p) dev_free(p, s); p = nullptr; }
    ~DevBuf() { reset(); }
    void *release() { void *q = p; p = nullptr; return q; }
};

// ---------------------------------------------------------------------------
// block tensors
// ---------------------------------------------------------------------------
constexpr int kMaxRank = ROSNET_MAX_RANK;
// Largest element count of a tensor: its two planes of 8-byte values,
// 2^62 bytes, and every byte offset into them stay within int64_t.
constexpr int64_t kMaxNumel = int64_t(1) << 58;

struct Layout {
    int rank = 0;
    int64_t shape[kMaxRank];
    int64_t block[kMaxRank];
    int64_t numel = 1;
    // element strides (within one plane) of the grid and intra-block index of
    // every axis in the block-major layout: offset(x) = sum_i (x_i / b_i) *
    // gstride[i] + (x_i % b_i) * lstride[i]
    int64_t gstride[kMaxRank];
    int64_t lstride[kMaxRank];
    void init(int r, const int64_t *sh, const int64_t *bl);  // validates, throws
};

}  // namespace rosnet

struct rosnet_btensor_s {
    rosnet::Layout lay;
    int dtype = 0;           // ROSNET_C64 / ROSNET_C128
    size_t elsize = 0;       // bytes of one real component (4 or 8)
    void *data = nullptr;    // real plane; imaginary plane at data + pstride*elsize
    int64_t pstride = 0;     // elements from the real to the imaginary plane
    cudaStream_t stream = nullptr;  // stream of the last write, for ordered free
    bool owned = true;       // false: a view of another tensor's storage
    void *re() const { return data; }
    void *im() const { return (char *)data + pstride * elsize; }
};

namespace rosnet {

// ---------------------------------------------------------------------------
// the GEMM view of a pairwise contraction (Sec. II-C steps 1-2)
// ---------------------------------------------------------------------------
// A fused index mode of one class (M: free in A, N: free in B, K:
// contracted) with its extent and element strides in the two tensors that
// carry it (M: A and C; N: B and C; K: A and B).
struct Mode {
    int64_t ext;
    int64_t s0, s1;
};

constexpr int kMaxModes = 2 * kMaxRank;

struct ModeList {
    int n = 0;
    Mode m[kMaxModes];      // outermost first
    int64_t total() const { int64_t t = 1; for (int i = 0; i < n; ++i) t *= m[i].ext; return t; }
};

struct GettView {
    ModeList M, N, K;
    int64_t Mtot = 1, Ntot = 1, Ktot = 1;
    bool a_m_fast = false;  // A's unit-stride mode is an M mode (else a K mode)
    bool b_n_fast = false;  // B's unit-stride mode is an N mode (else a K mode)
    bool c_n_fast = true;   // C's unit-stride mode is an N mode
};

// Build the view of C = tensordot(A, B, axes) for the three block layouts.
// axa/axb: contracted axis pairs; the caller has validated them.
GettView make_view(const Layout &A, const Layout &B, const Layout &C, int naxes,
                   const int *axa, const int *axb);

// Device-side problem descriptor of one pairwise contraction.  Offsets are
// in elements within a plane; the imaginary plane of a tensor starts
// *_plane elements after its real plane.
struct GettDesc {
    const void *a;
    const void *b;
    void *c;
    int64_t a_plane, b_plane, c_plane;
    const int64_t *offAM, *offCM, *offBN, *offCN, *offAK, *offBK;
    int64_t M, N, K;
    int64_t tiles_m, tiles_n;   // output tile grid of the kernel chosen for it
    int64_t tile_begin;         // first global CTA index of this problem in its launch
    void *part;                 // split-K partial sums [ksplit][2 planes][M*N], or NULL
    int32_t ksplit;             // number of contracted-index ranges (1 = no split)
    int32_t ktiles_per_split;   // k-tiles of each range
    int32_t flags;              // kFlag* bits
    int32_t kind;               // kernel family (KernelKind)
};

// CTAs of one problem in its launch (split-K ranges included)
inline int64_t desc_ctas(const GettDesc &d) { return d.tiles_m * d.tiles_n * (int64_t)d.ksplit; }

// Point a descriptor at its operands and result (honours kFlagSwapped).
inline void bind_operands(GettDesc &d, const void *A, const void *B, void *C, int64_t a_numel,
                          int64_t b_numel, int64_t c_numel);

enum : int32_t {
    kFlagAMFast = 1,
    kFlagBNFast = 2,
    kFlagCNFast = 4,
    kFlagSwapped = 8,   // roles of A and B exchanged (the kernel computes C^T = B^T A^T)
    kFlagAtomic = 16,   // split-K ranges add into C with atomics (C zeroed first)
    // A (B) is stored as a dense K x M (K x N) matrix in each plane: offAM[m]
    // = m and offAK[k] = k * M (offBN[n] = n, offBK[k] = k * N), so the packed
    // FP32 GEMM can load its tiles straight from it with TMA (no pack pass)
    kFlagADense = 32,
    kFlagBDense = 64,
    // packed FP32 GEMM: stream-K schedule (units of (tile, k-tile) split
    // evenly over one CTA per slot, partial tiles summed in a fixed order)
    kFlagStreamK = 128,
    // vector access for the low-arithmetic-intensity kernel (gett_gate_kernel):
    // A (B) along M (N) in runs of 8 contiguous elements whose offsets, and
    // those of every contracted index, are multiples of 4 (16-byte loads)
    kFlagAMVec = 256,
    kFlagBNVec = 512,
    // C along M (N) in runs of 8 contiguous elements, all offsets of the
    // other class multiples of 4
    kFlagCMVec = 1024,
    kFlagCNVec = 2048,
    // C with the N (M) index innermost and dense, and the innermost M (N)
    // mode right above it in runs of 8: 8 x N (8 x M) outputs are contiguous
    kFlagCNInner = 4096,
    kFlagCMInner = 8192,
};

// How the partial products of the matched block pairs of an output tile are
// summed (Sec. IV-A): automatic, one CTA over all pairs ("sequential"), split
// over CTAs with a fixed-order reduction of stored partials ("tree"), or split
// over CTAs adding into C in whatever order they finish ("commutative").
enum ReduceMode : int { kReduceAuto = 0, kReduceSequential = 1, kReduceTree = 2, kReduceCommutative = 3 };

enum KernelKind : int32_t {
    kKindSmall = 0,   // one thread per output, full K loop (low arithmetic intensity)
    kKindWarpK = 1,   // one warp per output, lanes split K, shuffle reduction
    kKindTiled = 2,   // 64x64 register-blocked tiles staged through shared memory
    kKindTiledWide = 3,  // 128x64 tiles (complex64 only), 8x4 outputs per thread
    kKindReduce = 4,     // sum of the split-K partials of a problem into C
    kKindTcTF32 = 5,     // tcgen05 tensor cores, TF32 products
    kKindTcTF32x3 = 6,   // tcgen05, 3 x TF32 split products
    kKindTcBF16x3 = 7,   // tcgen05, 3 x BF16 split products
    kKindZero = 8,       // zero C before a commutative (atomic) split-K launch
    kKindDot = 9,        // one CTA cluster per output, long K (e.g. a network's final scalar)
    kKindPackF32 = 10,   // plain FP32 on CUDA cores from packed operands (TMA-fed 64x64 tiles)
    kKindTiled256x16 = 11,  // 256x16 tiles (complex64 only): problems with few columns
    kKindTiled128x32 = 12,  // 128x32 tiles (complex64 only)
    kKindDirect = 13,       // 64x64 tiles, each CTA's K range (<= kDirectK) gathered in one pass
    kKindDirect256x16 = 14, // 256x16 tiles of the same kernel (complex64 only)
    kKindForest = 15,       // a plan's leaf-side small steps, one connected group per CTA
};

constexpr int kForestThreads = 512;    // threads of a gett_forest_kernel CTA
constexpr int kForestMaxSteps = 192;   // most steps of one fused group (its descriptors in shared memory)

constexpr int kDirectK = 32;   // longest contraction range of one direct-kernel CTA

// Low-arithmetic-intensity kinds (gett_gate_kernel): K and N in {1, 2, 4},
// M large; kind = kKindGateBase + 3 log2 K + log2 N.  Each thread takes
// gate_rows(kind) consecutive m.
constexpr int kKindGateBase = 16;
inline bool is_gate_kind(int kind) { return kind >= kKindGateBase && kind < kKindGateBase + 9; }
inline int gate_log2(int64_t x) { return x == 1 ? 0 : x == 2 ? 1 : x == 4 ? 2 : -1; }
inline int gate_rows(int kind) {
    const int lk = (kind - kKindGateBase) / 3, ln = (kind - kKindGateBase) % 3;
    return lk + ln >= 3 ? 4 : 8;   // fewer rows per thread when K * N >= 8 (registers)
}

inline bool is_direct_kind(int kind) { return kind == kKindDirect || kind == kKindDirect256x16; }
// CTA tile of a direct kind, and whether it applies to a problem
inline void direct_tile(int kind, int *bm, int *bn) {
    if (kind == kKindDirect256x16) { *bm = 256; *bn = 16; }
    else { *bm = 64; *bn = 64; }
}
inline bool direct_kind_ok(int kind, int dtype, int64_t M, int64_t N) {
    if (kind == kKindDirect) return true;
    return kind == kKindDirect256x16 && dtype == ROSNET_C64 && M >= 128;
}

// Register-tiled CUDA-core kinds (gett_tiled_kernel), their CTA tile, and
// whether one applies to a problem of dtype and (M, N).
inline bool is_tiled_kind(int kind) {
    return kind == kKindTiled || kind == kKindTiledWide || kind == kKindTiled256x16 || kind == kKindTiled128x32;
}
inline void tiled_tile(int kind, int *bm, int *bn) {
    switch (kind) {
        case kKindTiledWide: *bm = 128; *bn = 64; break;
        case kKindTiled256x16: *bm = 256; *bn = 16; break;
        case kKindTiled128x32: *bm = 128; *bn = 32; break;
        default: *bm = 64; *bn = 64; break;
    }
}
inline bool tiled_kind_ok(int kind, int dtype, int64_t M, int64_t N) {
    if (kind == kKindTiled) return true;
    if (dtype != ROSNET_C64) return false;
    if (kind == kKindTiledWide) return M >= 128 && N >= 48;
    if (kind == kKindTiled256x16) return M >= 128;
    if (kind == kKindTiled128x32) return M >= 64;
    return false;
}

// Kinds that run as pack kernels + a GEMM on packed operands held in a
// per-problem workspace (one launch sequence per problem), and their packed
// mode: 0 TF32, 1 3xTF32, 2 3xBF16 (tcgen05), 3 FP32 (CUDA cores).
constexpr int kPackedModeF32 = 3;
inline bool is_packed_kind(int kind) {
    return (kind >= kKindTcTF32 && kind <= kKindTcBF16x3) || kind == kKindPackF32;
}
inline int packed_mode(int kind) { return kind == kKindPackF32 ? kPackedModeF32 : kind - kKindTcTF32; }

constexpr int kDotCTAs = 8;   // CTAs of the cluster that computes one output of the dot kernel

inline void bind_operands(GettDesc &d, const void *A, const void *B, void *C, int64_t a_numel,
                          int64_t b_numel, int64_t c_numel) {
    if (d.flags & kFlagSwapped) {
        d.a = B; d.b = A; d.a_plane = b_numel; d.b_plane = a_numel;
    } else {
        d.a = A; d.b = B; d.a_plane = a_numel; d.b_plane = b_numel;
    }
    d.c = C;
    d.c_plane = c_numel;
}

// Bytes of split-K partials a problem needs (0 without split).
size_t desc_part_bytes(const GettDesc &d, int dtype);

// Offsets tables: 2*M + 2*N + 2*K int64 entries, built on the device.
size_t table_entries(const GettView &v);
void launch_build_tables(const GettView &v, int64_t *tables, cudaStream_t s);
void fill_desc_tables(GettDesc &d, const GettView &v, const int64_t *tables);

// The large index class of a low-arithmetic-intensity problem (a gate kind)
// needs no offset table: the kernel computes its offsets from a mode record
// [n, (extent, stride in the first tensor, stride in the second) x n],
// outermost mode first.  A table layout puts one class (record_class: 0 M,
// 1 N; -1 none) as such a record and the others as tables.
struct TableLayout {
    int record_class = -1;
    int64_t off[3] = {0, 0, 0};   // entry offset of the M, N and K parts
    int64_t entries = 0;
};
inline int64_t record_entries(const ModeList &ml) { return 1 + 3 * (int64_t)ml.n; }
void host_mode_record(const ModeList &ml, int64_t *out);
TableLayout table_layout(const GettView &v, int record_class);
void launch_build_tables(const GettView &v, const TableLayout &L, int64_t *tables, cudaStream_t s);
// The class a problem keeps as a mode record: the one the gate kernel walks
// when the kernel choice for the view (with `clear_flags` removed, e.g. the
// vector flags of operands whose address changes between calls) is a gate
// kind, else -1.
int gate_record_class(const GettView &v, int dtype, int precision, int reduce_mode, int clear_flags);
// The same with the M, N and K tables ([offsets in the first tensor | in the
// second] of each class) at separate addresses.
void fill_desc_tables(GettDesc &d, const GettView &v, const int64_t *tm, const int64_t *tn,
                      const int64_t *tk);

// Choose the kernel family, tile grid and split-K for a problem (may swap
// the operand roles; call bind_operands afterwards).
void choose_kernel(GettDesc &d, int dtype, int precision, int reduce_mode = kReduceAuto);
int check_reduce(const rosnet_opts *opts);
inline int64_t zero_ctas(const GettDesc &d) { return (d.M * d.N + 1023) / 1024; }

// Launch one group of problems of the same kind and dtype.  `descs` is in
// device memory (ndesc entries, with tile_begin prefix sums); total_tiles is
// the sum of tiles_m*tiles_n.
// The fused leaf-side small steps of a plan (gett_forest_kernel): `ctas`
// groups, program `prog` in device memory.
void launch_forest(int dtype, const GettDesc *descs, const int64_t *prog, int64_t ctas, cudaStream_t s);
void launch_gett_group(int kind, int dtype, const GettDesc *descs, int ndesc,
                       int64_t total_tiles, cudaStream_t s);

// Pack/unpack between dense row-major interleaved and block-major planar
// (imaginary plane `pstride` elements after the real one).  Pack covers the
// dense row-major entries [start, start + count) of the tensor.
void launch_pack(const Layout &lay, int dtype, const void *dense_interleaved, void *planar,
                 int64_t pstride, int64_t start, int64_t count, cudaStream_t s);
void launch_unpack(const Layout &lay, int dtype, const void *planar, int64_t pstride,
                   void *dense_interleaved, cudaStream_t s);

// Copy src (block-major planar) to dst with a different block shape and/or
// axis permutation: dst axis i = src axis perm[i].
void launch_relayout(const Layout &src, const Layout &dst, const int *perm, int dtype,
                     const void *src_planar, int64_t src_pstride, void *dst_planar,
                     int64_t dst_pstride, cudaStream_t s);

// Create / free tensors.
rosnet_btensor new_tensor(int rank, const int64_t *shape, const int64_t *block, int dtype,
                          cudaStream_t s);
void free_tensor(rosnet_btensor t);

// One pairwise contraction enqueued on s into an existing C (used by both
// rosnet_tensordot and the network executor).  workspace for the tables is
// allocated from the allocator.
void tensordot_into(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axa,
                    const int *axb, rosnet_btensor C, int precision, cudaStream_t s,
                    int reduce_mode = kReduceAuto);

}  // namespace rosnet
