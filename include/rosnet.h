/*
 * rosnet.h -- C ABI of the B300 block tensor library (librosnet.so).
 *
 * The library computes the blocked pairwise tensordot of the RosneT paper
 * (Sanchez-Ramirez et al., "RosneT: A Block Tensor Algebra Library for
 * Out-of-Core Quantum Computing Simulation"):
 *
 *   - a block tensor is a tensor cut into a uniform grid of equally shaped
 *     blocks (Sec. II-C, "Dimension Extents" layout);
 *   - the pairwise contraction C[fA, fB] = sum_k A[fA, k] B[k, fB] of Sec. II-A
 *     is computed per output block as the sum, over the pairs of A and B blocks
 *     matched on the contracted-index block coordinates, of the local
 *     contraction of each pair (Sec. II-C steps 1-4); the order of that sum is
 *     free (Sec. IV-A, commutative reduction);
 *   - a tensor network (e.g. a quantum circuit, Sec. II-A) is contracted as a
 *     sequence of such pairwise contractions.
 *
 * Conventions shared by every call
 * --------------------------------
 *   * Element types: complex64 (two float32) or complex128 (two float64).
 *   * Host buffers passed to upload/download are DENSE, ROW-MAJOR and
 *     INTERLEAVED (re, im, re, im, ...), i.e. numpy's C-order complex arrays.
 *   * Device storage is owned by the library: block-major (all blocks laid out
 *     one after another in row-major order of their grid coordinates, each
 *     block row-major inside) and planar (all real parts, then all imaginary
 *     parts).  Callers never need to know this layout.
 *   * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is enqueued on that stream; calls
 *     return without waiting for it unless stated otherwise.  Errors raised by
 *     kernels after a call has returned are reported by rosnet_sync().
 *   * Every call returns a rosnet_status (0 = ROSNET_OK, negative = error).
 *     No C++ exception crosses the ABI.  On error, output handles are set to
 *     NULL and nothing is leaked.  Handles returned by create / tensordot /
 *     contract belong to the caller, who must pass them to
 *     rosnet_btensor_destroy.  Input handles are never modified or freed.
 *   * The library is for one GPU: it uses the CUDA device that is current on
 *     the calling thread.
 */
#ifndef ROSNET_H
#define ROSNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- */
/* status codes                                                             */
/* ----------------------------------------------------------------------- */
typedef int rosnet_status;
#define ROSNET_OK                  0
#define ROSNET_ERR_INVALID_ARG    -1  /* NULL handle/pointer, bad axis, bad enum   */
#define ROSNET_ERR_SHAPE          -2  /* extents of contracted axes differ, bad shape */
#define ROSNET_ERR_BLOCK_MISMATCH -3  /* block extent does not divide the extent, or
                                         contracted axes have different block extents */
#define ROSNET_ERR_DTYPE          -4  /* operands of different element types        */
#define ROSNET_ERR_ALLOC          -5  /* the allocator returned NULL                 */
#define ROSNET_ERR_RANK_LIMIT     -6  /* rank > ROSNET_MAX_RANK                       */
#define ROSNET_ERR_CUDA           -7  /* a CUDA runtime call failed                   */
#define ROSNET_ERR_TIMEOUT        -8  /* a bounded device-side wait gave up           */
#define ROSNET_ERR_UNSUPPORTED    -9  /* e.g. a precision mode for the wrong dtype    */

/* Tensors of any rank from 0 to ROSNET_MAX_RANK are accepted (the paper
 * needs more than numpy's 32 dimensions, Sec. V). */
#define ROSNET_MAX_RANK 64

typedef enum {
    ROSNET_C64 = 1,   /* complex64: float32 real and imaginary parts  */
    ROSNET_C128 = 2   /* complex128: float64 real and imaginary parts */
} rosnet_dtype;

/* Arithmetic used for the block products (the sum is always accumulated in
 * at least float32; see each mode).  The tensor-core modes apply to block
 * products large enough to fill a 128 x 128 tile; smaller products of the same
 * call use the FP32 CUDA-core kernels. */
typedef enum {
    ROSNET_PREC_DEFAULT = 0, /* FP32 CUDA cores for C64, FP64 for C128            */
    ROSNET_PREC_FP32 = 1,    /* C64 only: float32 products and sums (CUDA cores)  */
    ROSNET_PREC_TF32 = 2,    /* C64 only: TF32 tensor-core products (operands
                                rounded to 10-bit mantissas), FP32 sums           */
    ROSNET_PREC_BF16X3 = 3,  /* C64 only: each float32 operand split into bf16
                                hi + lo; hi*hi + hi*lo + lo*hi on tensor cores,
                                FP32 sums                                         */
    ROSNET_PREC_FP64 = 4,    /* C128 only: float64 products and sums              */
    ROSNET_PREC_TF32X3 = 5   /* C64 only: each float32 operand split into TF32
                                big + small; big*big + big*small + small*big on
                                tensor cores, FP32 sums                           */
} rosnet_precision;

typedef struct rosnet_btensor_s *rosnet_btensor;

/* Options of tensordot/contract (pass NULL for defaults: all fields 0). */
typedef struct {
    int32_t precision;          /* a rosnet_precision                                */
    int32_t flags;              /* ROSNET_OPT_* bits                                 */
    int64_t max_block_entries;  /* contract only: if > 0, every intermediate whose
                                   block holds more entries is re-blocked by turning
                                   its slowest-varying axes into grid axes until the
                                   block fits (0 = blocks inherited from operands)  */
    int64_t reserved[6];        /* must be 0                                         */
} rosnet_opts;

#define ROSNET_OPT_GRAPH  0x1   /* contract: capture the step sequence in a CUDA
                                   graph on first use and replay it afterwards      */
#define ROSNET_OPT_NOGROUP 0x2  /* contract: one launch per step instead of one
                                   grouped launch per dependency wave               */
/* How the partial products of the B_k matched block pairs of an output tile
 * are summed (Sec. IV-A).  At most one; none = chosen per problem (split only
 * when the output tiles cannot fill the GPU, tree-reduced).
 *   SEQUENTIAL   one CTA loops over every pair of its tile (no split);
 *   TREE         pairs split over CTAs, partial tiles stored, then summed in
 *                a fixed order (deterministic);
 *   COMMUTATIVE  pairs split over CTAs, each adding into C as it finishes
 *                (order-free, no partial storage, not bitwise reproducible). */
#define ROSNET_OPT_REDUCE_SEQUENTIAL  0x10
#define ROSNET_OPT_REDUCE_TREE        0x20
#define ROSNET_OPT_REDUCE_COMMUTATIVE 0x40
#define ROSNET_OPT_AUTOTUNE 0x80 /* contract: when planning, time the candidate
                                   CUDA-core kernels (tile shape, contracted-range
                                   split) of every step with >= 1e8 flops on the
                                   plan's own operands and keep the fastest;
                                   choices are cached per (dtype, M, N, K, access
                                   pattern) for the process                       */
#define ROSNET_OPT_TIMING 0x4   /* contract: record CUDA events around the plan's
                                   heaviest launch (most 8*M*N*K flops) on the
                                   call's stream; read with rosnet_timing_drain    */

/* ----------------------------------------------------------------------- */
/* memory                                                                   */
/* ----------------------------------------------------------------------- */
/*
 * Replace the device allocator.  alloc(bytes, stream, ctx) must return device
 * memory usable in stream order on `stream` (or NULL on failure); free(ptr,
 * stream, ctx) releases it in stream order.  Passing alloc = free = NULL
 * restores the built-in allocator (cudaMallocAsync / cudaFreeAsync on the
 * device's default memory pool, which then keeps freed memory for reuse).
 * A block is always freed by the allocator that made it, so switching to a
 * different allocator while library blocks are outstanding (tensors, cached
 * plans) returns INVALID_ARG.  Not thread-safe with concurrent calls.
 */
rosnet_status rosnet_set_allocator(void *(*alloc)(size_t bytes, void *stream, void *ctx),
                                   void (*free)(void *ptr, void *stream, void *ctx),
                                   void *ctx);

/* Device blocks the library has requested from its allocator since load
 * (*requests) and those not yet freed (*live); either pointer may be NULL. */
rosnet_status rosnet_alloc_stats(int64_t *requests, int64_t *live);

/* ----------------------------------------------------------------------- */
/* block tensors (Sec. II-C)                                                */
/* ----------------------------------------------------------------------- */
/*
 * Create an uninitialised block tensor of `rank` axes with extents shape[i]
 * and block extents block_shape[i] (block_shape may be NULL: one block).
 * Each block_shape[i] must be >= 1 and divide shape[i]; the grid extent of
 * axis i is shape[i] / block_shape[i].  Device memory (numel * element size)
 * comes from the allocator in stream order on `stream`.
 * Errors: INVALID_ARG (out == NULL, shape == NULL with rank > 0, extent < 0),
 * SHAPE (more than 2^58 elements), RANK_LIMIT, BLOCK_MISMATCH, DTYPE, ALLOC.
 */
rosnet_status rosnet_btensor_create(int rank, const int64_t *shape, const int64_t *block_shape,
                                    rosnet_dtype dtype, void *stream, rosnet_btensor *out);

/* Release a tensor (stream-ordered on the stream it was created or last
 * written on).  NULL is accepted and ignored. */
rosnet_status rosnet_btensor_destroy(rosnet_btensor t);

/*
 * Copy a dense row-major interleaved host array (numel complex values of the
 * tensor's dtype) into the tensor.  The host buffer may be pageable or pinned;
 * it is read before the call returns if pageable, or in stream order if it is
 * pinned (the caller must keep it alive until the stream reaches the copy).
 */
rosnet_status rosnet_btensor_upload(rosnet_btensor t, const void *host, void *stream);

/*
 * Copy `count` complex values, the dense row-major entries [start, start +
 * count) of the tensor, from a host buffer into the tensor (e.g. to fill a
 * tensor larger than host memory in pieces).  Same rules as
 * rosnet_btensor_upload; INVALID_ARG if the range is outside the tensor.
 */
rosnet_status rosnet_btensor_upload_range(rosnet_btensor t, const void *host, int64_t start,
                                          int64_t count, void *stream);

/*
 * A view of t with its first nfix axes fixed to values[0..nfix): the
 * projection of those indices onto one basis state each (Sec. II-B, slicing,
 * which the paper reads as a block division).  Each fixed axis must be a grid
 * axis (block extent 1), so the view is a contiguous run of t's blocks and
 * shares t's storage: no copy is made.  The view has rank - nfix axes with
 * t's remaining extents and block extents; it must be destroyed before t, and
 * writes through it (upload) change t.  Errors: INVALID_ARG (index out of
 * range), BLOCK_MISMATCH (a fixed axis with block extent > 1).
 */
rosnet_status rosnet_btensor_slice(rosnet_btensor t, int nfix, const int64_t *values,
                                   rosnet_btensor *view);

/*
 * A view of one block of t (grid_coords[i] in [0, shape[i] / block_shape[i])):
 * a tensor whose shape is t's block shape, sharing t's storage (a block is
 * contiguous in the block-major layout, so this is the unit to move between
 * device and host).  Destroy it before t.  Errors: INVALID_ARG.
 */
rosnet_status rosnet_btensor_block(rosnet_btensor t, const int64_t *grid_coords, rosnet_btensor *view);

/*
 * A view of t with axes[j] fixed to values[j] for j < nfix (any axes, any
 * block extents): the projection of those indices on one basis state each,
 * i.e. the slicing of those bonds (Sec. II-B).  The view keeps t's strides
 * for the remaining axes (it need not be contiguous), shares t's storage and
 * must be destroyed before t.  Errors: INVALID_ARG (repeated or bad axis,
 * value out of range).
 */
rosnet_status rosnet_btensor_fix(rosnet_btensor t, int nfix, const int *axes, const int64_t *values,
                                 rosnet_btensor *view);

/* Copy the tensor into a dense row-major interleaved host array.  Blocks
 * until the data is on the host (synchronises `stream`). */
rosnet_status rosnet_btensor_download(rosnet_btensor t, void *host, void *stream);

/* As rosnet_btensor_download, but only enqueued on `stream` (no wait): the
 * host buffer must stay valid, and is complete once the stream reaches this
 * point; with page-locked host memory the copy overlaps other work. */
rosnet_status rosnet_btensor_download_async(rosnet_btensor t, void *host, void *stream);

/*
 * Copy the raw storage of a tensor that owns it -- 2 * numel elements of its
 * dtype's real type: the real plane, then the imaginary plane, each in the
 * tensor's block-major element order (plain row-major for a one-block
 * tensor) -- from / to host memory (or device memory of the same GPU: the
 * copy direction follows the pointer), enqueued on `stream` without waiting,
 * one copy and no kernel.  The buffer must stay valid until the stream
 * reaches this point; page-locked memory lets the copy overlap other work.
 * INVALID_ARG for NULL arguments, UNSUPPORTED for views (slice / fix /
 * block), whose storage belongs to another tensor.
 */
rosnet_status rosnet_btensor_upload_raw(rosnet_btensor t, const void *host, void *stream);
rosnet_status rosnet_btensor_download_raw(rosnet_btensor t, void *host, void *stream);

/* Shape, block shape (arrays of at least `rank` entries; either may be NULL)
 * and dtype (may be NULL) of a tensor.  *rank is always written. */
rosnet_status rosnet_btensor_info(rosnet_btensor t, int *rank, int64_t *shape,
                                  int64_t *block_shape, rosnet_dtype *dtype);

/* Device addresses of the real and imaginary planes (block-major layout);
 * for callers that move blocks themselves.  Either output may be NULL. */
rosnet_status rosnet_btensor_planes(rosnet_btensor t, void **re, void **im);

/* ----------------------------------------------------------------------- */
/* pairwise blocked tensordot (Sec. II-A, II-C, IV-A)                       */
/* ----------------------------------------------------------------------- */
/*
 * C = tensordot(A, B, axes=(axes_a, axes_b)) with numpy's conventions: axis
 * axes_a[i] of A is contracted with axis axes_b[i] of B; C's axes are A's free
 * axes in order followed by B's free axes in order; naxes = 0 is the outer
 * product; contracting every axis gives a rank-0 tensor (one value).
 * Block rules (Sec. II-C): contracted pairs must have equal extents (else
 * SHAPE) and equal block extents (else BLOCK_MISMATCH); C's block extents are
 * those of the free axes, so an output block is the sum over the B_k matched
 * block pairs.  A and B must have the same dtype (else DTYPE); opts->precision
 * must suit it (else UNSUPPORTED).  *out_C is a new tensor owned by the caller.
 */
rosnet_status rosnet_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes,
                               const int *axes_a, const int *axes_b,
                               const rosnet_opts *opts, void *stream, rosnet_btensor *out_C);

/*
 * rosnet_tensordot_noalloc -- the same contraction as rosnet_tensordot for
 * callers that cannot allocate device memory at the call (the paper has no
 * counterpart: it is an interface convenience of this library).  Callers in
 * this position include code running inside a framework that owns all device
 * memory and forbids foreign allocations, real-time or embedded code with a
 * fixed memory budget committed up front, and paths where an allocation could
 * block or fail unpredictably.
 *
 * The caller passes the operands and an already created output tensor C whose
 * shape, block shape and dtype are those rosnet_tensordot would give the
 * result (else SHAPE / BLOCK_MISMATCH / DTYPE).  C's storage must not overlap
 * A's or B's: the byte range from a tensor's data pointer to the end of its
 * imaginary plane is compared, so a view of an operand's storage is refused
 * like the operand itself (INVALID_ARG).  The call allocates nothing: the
 * offset tables, split-K partial sums and packed operands of the tensor-core
 * and packed-FP32 kernels are placed in one fixed device array of
 * ROSNET_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that
 * loads the library keeps until the process exits.  When the kernel choice
 * of rosnet_tensordot would split the contracted range over CTAs with partial
 * sums that do not fit (and no reduction flag asks for the split), the call
 * runs unsplit instead; a problem that still needs more scratch is rejected
 * with ROSNET_ERR_UNSUPPORTED before anything is launched (rosnet_last_error()
 * gives the bytes needed).  opts as rosnet_tensordot:
 * the precision and the reduction flags are honoured; ROSNET_OPT_AUTOTUNE is
 * refused (UNSUPPORTED), because timing candidate kernels needs buffers of
 * their own.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset() on a device the entry point must not be used on it again.
 * All calls share the array and it keeps the previous call's contents; every
 * byte a call reads from it is written earlier by the same call, so nothing
 * needs clearing, but calls that overlap on the GPU (on different streams, or
 * from different threads) race on it: serialise them.  Errors as
 * rosnet_tensordot.
 */
#define ROSNET_NOALLOC_SCRATCH_BYTES (4u << 20)
rosnet_status rosnet_tensordot_noalloc(rosnet_btensor A, rosnet_btensor B, int naxes,
                                       const int *axes_a, const int *axes_b, rosnet_btensor C,
                                       const rosnet_opts *opts, void *stream);

/*
 * Out-of-core tensordot (the paper's out-of-core premise, Sec. I and III: data
 * larger than memory lives on the next storage tier and only task-sized pieces
 * are resident).  C = tensordot(A, B, axes) is computed in output chunks along
 * A's first `nsplit` axes, which must be free grid axes (block extent 1):
 * chunk c fixes them to the row-major digits of c (c in [0, prod of their
 * extents)), i.e. it is tensordot(slice of A, B), a contiguous run of C's
 * blocks.  Chunks first_chunk .. first_chunk + nchunks - 1 are computed into
 * two alternating device buffers and each is copied, on a side stream while
 * the next one is computed, to host_out: slot (c - first_chunk) % nslots with
 * nslots = host_bytes / chunk_bytes, chunk_bytes = 2 * chunk entries *
 * element size, in the raw block-major planar layout (real plane, then
 * imaginary plane).  host_out should be pinned for the copies to overlap.
 * Returns when every copy has completed.  Errors as rosnet_tensordot, plus
 * INVALID_ARG (bad chunk range, host buffer smaller than one chunk) and
 * BLOCK_MISMATCH (a split axis with block extent > 1).
 */
rosnet_status rosnet_tensordot_ooc(rosnet_btensor A, rosnet_btensor B, int naxes,
                                   const int *axes_a, const int *axes_b, int nsplit,
                                   int64_t first_chunk, int64_t nchunks, const rosnet_opts *opts,
                                   void *host_out, size_t host_bytes, void *stream);

/*
 * The same with A left in host memory (the out-of-core tier for an operand
 * larger than the device memory, Sec. I and III): A is described by its rank,
 * shape and block shape (NULL block_a: one block), has B's dtype, and lives at
 * a_host in the raw block-major planar layout (the real plane, then the
 * imaginary plane, numel elements each: what rosnet_btensor_download_raw
 * writes).  Chunk c needs only its slice of A (the split axes fixed: one
 * contiguous run of blocks per plane), which is copied into one of two
 * device buffers on an input stream while the previous chunk is computed;
 * output chunks stream out as in rosnet_tensordot_ooc.  B stays on the
 * device.  a_host and host_out should be pinned for the copies to run
 * asynchronously; the caller keeps a_host unchanged until the call returns.
 * Device memory used: two slices of A, two output chunks and B.  Errors as
 * rosnet_tensordot_ooc, plus INVALID_ARG for a NULL a_host (unless A is
 * empty or nchunks is 0) and the layout errors of rosnet_btensor_create.
 */
rosnet_status rosnet_tensordot_ooc_host(int rank_a, const int64_t *shape_a, const int64_t *block_a,
                                        const void *a_host, rosnet_btensor B, int naxes,
                                        const int *axes_a, const int *axes_b, int nsplit,
                                        int64_t first_chunk, int64_t nchunks,
                                        const rosnet_opts *opts, void *host_out, size_t host_bytes,
                                        void *stream);

/* ----------------------------------------------------------------------- */
/* networks (Sec. II-A)                                                     */
/* ----------------------------------------------------------------------- */
/*
 * A tensor network: tensor t has ranks[t] axes labelled labels[t][0..ranks[t]).
 * A label carried by two tensors is a bond and is summed over when they are
 * joined, unless it appears in out_labels; out_labels (nout entries, each
 * carried by exactly one tensor) stay open and give the result's axis order.
 * Labels are arbitrary int64 values; every tensor must share the dtype.
 */
typedef struct {
    int32_t ntensors;
    const rosnet_btensor *tensors;
    const int32_t *ranks;
    const int64_t *const *labels;
    int32_t nout;
    const int64_t *out_labels;
} rosnet_network;

/*
 * A contraction path in SSA form: step s joins the tensors with ids
 * pairs[2s] and pairs[2s+1] and creates id ntensors + s.  A full path has
 * ntensors - 1 steps.
 */
typedef struct {
    int32_t nsteps;
    const int32_t *pairs;
} rosnet_path;

/*
 * Rank reduction before path search (the paper builds and simplifies its
 * circuit networks with a front end before choosing a path, Sec. V): while
 * some tensor of rank <= max_rank (0, 1 or 2) not marked in keep shares a
 * label with a tensor not marked in keep, it is absorbed into such a
 * neighbour -- the one of highest rank, then lowest index -- by one
 * rosnet_tensordot on `stream` with `opts` (precision as that call).  Only
 * labels carried by exactly these two tensors are summed (a label in
 * out_labels never is); the merged tensor's labels are the neighbour's
 * remaining labels, then the absorbed tensor's, and it takes the
 * neighbour's position.  Tensors marked in keep (e.g. output projectors that
 * change from query to query) are neither absorbed nor absorbed into.
 *
 * Output, survivors in input order: tensors_out[0 .. *ntensors_out), their
 * ranks, their labels concatenated in labels_out, and origin_out[i] = the
 * input index whose position survivor i holds.  tensors_out, ranks_out and
 * origin_out must hold ntensors entries and labels_out the total rank of the
 * input (the total never grows).  A survivor that absorbed nothing is the
 * caller's own handle; every other one is a new tensor owned by the caller
 * (release it with rosnet_btensor_destroy).  The absorbed input tensors are
 * not modified.  keep may be NULL (nothing kept).  Errors: INVALID_ARG
 * (NULL outputs, max_rank outside 0..2, a rank that does not match its
 * tensor), and the errors of rosnet_tensordot, after which no new tensor is
 * left alive.
 */
rosnet_status rosnet_simplify(const rosnet_network *net, const uint8_t *keep, int32_t max_rank,
                              const rosnet_opts *opts, void *stream, rosnet_btensor *tensors_out,
                              int32_t *ranks_out, int64_t *labels_out, int32_t *origin_out,
                              int32_t *ntensors_out);

/*
 * A greedy min-size path (the paper takes its paths from an external path
 * optimiser, Sec. V; this one is the library's own): at each step join the
 * pair of tensors sharing at least one label whose result is smallest; ties go
 * to the smaller size(result) - size(a) - size(b), then to the lowest ids;
 * disconnected pieces are joined last by outer products.  pairs_out must hold
 * 2 * (ntensors - 1) ints; *nsteps receives ntensors - 1.  Host-only.
 */
rosnet_status rosnet_path_greedy(const rosnet_network *net, int32_t *pairs_out, int32_t *nsteps);

/* The same greedy path from labels and extents alone (no tensors, no GPU):
 * tensor t has ranks[t] axes with labels[t][i] and extents extents[t][i].
 * Errors: INVALID_ARG, SHAPE (a label with two extents), UNSUPPORTED (a label
 * on more than two tensors), RANK_LIMIT. */
rosnet_status rosnet_path_greedy_extents(int32_t ntensors, const int32_t *ranks,
                                         const int64_t *const *labels,
                                         const int64_t *const *extents, int32_t nout,
                                         const int64_t *out_labels, int32_t *pairs_out,
                                         int32_t *nsteps);

/*
 * A cheaper path by randomized greedy search (the paper takes its paths from
 * an external optimiser, Sec. V): trial 0 is rosnet_path_greedy_extents;
 * every further trial joins, at each step, the connected pair with the
 * smallest size(result) - size(a) - size(b) perturbed by Gumbel noise of
 * relative scale `temperature`; the path with the fewest total 8*M*N*K flops
 * wins (*flops, may be NULL).  Deterministic for a given seed.  Host-only.
 */
rosnet_status rosnet_path_search(int32_t ntensors, const int32_t *ranks,
                                 const int64_t *const *labels, const int64_t *const *extents,
                                 int32_t nout, const int64_t *out_labels, int32_t ntrials,
                                 uint64_t seed, double temperature, int32_t *pairs_out,
                                 int32_t *nsteps, double *flops);

/*
 * Bonds to slice (Sec. II-B): greedily, nslice times, the bond whose slicing
 * gives the smallest (largest intermediate, total flops over all slices) for
 * the given path.  chosen[0..nslice) receives the labels; *max_entries the
 * largest intermediate of one slice, *flops the total over all slices (either
 * may be NULL).  Host-only.  INVALID_ARG if the path is not a valid SSA path
 * of ntensors - 1 steps (an id out of range, reused, or paired with itself)
 * or nslice exceeds the number of bonds.
 */
rosnet_status rosnet_slice_search(int32_t ntensors, const int32_t *ranks,
                                  const int64_t *const *labels, const int64_t *const *extents,
                                  int32_t nout, const int64_t *out_labels, int32_t nsteps,
                                  const int32_t *pairs, int32_t nslice, int64_t *chosen,
                                  double *max_entries, double *flops);

/*
 * Contract a network along a path; *out is a new tensor whose axes follow
 * out_labels (rank 0 for a closed network such as one amplitude).
 * Intermediates live in one device arena sized from their lifetimes.  With
 * ROSNET_OPT_GRAPH the launch sequence is captured in a CUDA graph, keyed by
 * the network's structure (shapes, labels, path, options), and replayed on
 * later calls with the same structure.  Errors as rosnet_tensordot, plus
 * INVALID_ARG for a malformed path or labels.
 */
rosnet_status rosnet_contract(const rosnet_network *net, const rosnet_path *path,
                              const rosnet_opts *opts, void *stream, rosnet_btensor *out);

/*
 * Elapsed device time of the heaviest launch of every rosnet_contract call
 * made with ROSNET_OPT_TIMING since the last drain (oldest first, at most the
 * newest 4096).  Waits for those events.  The heaviest launch is the one with
 * the most algorithmic work.  ms[i] receives the milliseconds of its GEMM
 * kernel (for a packed-operand launch -- tensor-core or packed FP32 -- after
 * the operand packs) and ms_whole[i] those of the whole launch, operand packs
 * included (the same for launches without packs); ms_whole, flops, bytes and
 * kinds may be NULL.  flops[i] / bytes[i] / kinds[i] receive the launch's
 * algorithmic work -- sum of 8*M*N*K and of
 * (|A| + |B| + |C|) * element size over its problems -- and its kernel family
 * (2 = 64x64 tiles, 3 = 128x64, 11 = 256x16, 12 = 128x32, 13 / 14 = direct
 * short-range tiles, 5-7 = tcgen05 TF32 / 3xTF32 / 3xBF16, 10 = packed FP32;
 * others are the small-problem kernels).  *n receives the
 * number of entries written (<= max_entries).
 */
rosnet_status rosnet_timing_drain(double *ms, double *ms_whole, double *flops, double *bytes,
                                  int32_t *kinds, int32_t max_entries, int32_t *n);

/*
 * Autotuner decisions (ROSNET_OPT_AUTOTUNE) as text, so that a later process
 * can plan with the same kernels without timing them again.  One line per
 * tuned problem shape, eight integers separated by spaces:
 *     dtype key_flags M N K kind ksplit schedule
 * (kind: 2 = 64x64 tiles, 3 = 128x64, 11 = 256x16, 12 = 128x32, 13 / 14 =
 * direct 64x64 / 256x16 (one 32-long contracted range per CTA, so ksplit =
 * ceil(K / 32)), 10 = packed FP32; ksplit = number of contracted-index
 * ranges, 1 = none; schedule = 1 for the packed FP32 GEMM's stream-K
 * schedule, else 0; a line without it is read with schedule 0).
 * rosnet_tune_export writes the text, NUL-terminated, into buf when cap is
 * large enough; *len always receives the bytes needed (terminator included).
 * rosnet_tune_import merges the lines of a NUL-terminated text into the
 * table (later entries replace earlier ones of the same shape).  Every entry
 * is checked against its shape first; INVALID_ARG (and nothing merged) for a
 * malformed line, an unknown kind or dtype, or a split a problem of that
 * shape cannot have.  Neither call touches the device.
 */
rosnet_status rosnet_tune_export(char *buf, size_t cap, size_t *len);
rosnet_status rosnet_tune_import(const char *text);

/* Free every cached contraction plan (arena, offset tables, descriptors,
 * CUDA graph).  Plans are cached by rosnet_contract and kept until this call;
 * the caller must make sure no contraction is still running. */
rosnet_status rosnet_release_plans(void);

/*
 * Keep at most max_plans cached contraction plans (0: no limit, the
 * default; a negative value leaves the limit as it is, to query).  When a new
 * plan would exceed the limit, the least recently used plans are freed
 * first; lowering the limit frees the excess at once.  Work that a freed plan
 * already enqueued completes normally (its device buffers are released in
 * stream order, a graph still running is freed when it completes); its
 * undrained timing records are dropped.  A later call with a freed plan's
 * structure plans it again.  *cached (may be NULL) receives the number of
 * cached plans after the call.  Host-side; never fails on valid input.
 */
rosnet_status rosnet_plan_cache_limit(int32_t max_plans, int32_t *cached);

/*
 * Contract nnet networks (each with its own path, as rosnet_contract) in one
 * plan: the steps of all networks that sit at the same dependency depth run
 * in the same grouped launches, and a step whose operands and contraction are
 * identical to one already planned (same operand tensors -- same storage and
 * layout -- same contracted axes, same result blocks) is computed once and
 * shared.  Slices of one network (Sec. II-B) share every step that no sliced
 * bond reaches, so their common work is done once.  outs[i] receives network
 * i's result (new tensors owned by the caller).  Networks must share a dtype.
 * Options and errors as rosnet_contract.
 */
rosnet_status rosnet_contract_batch(int32_t nnet, const rosnet_network *nets,
                                    const rosnet_path *paths, const rosnet_opts *opts,
                                    void *stream, rosnet_btensor *outs);

/* For a batch already planned (same arguments as rosnet_contract_batch): the
 * number of path steps requested, of distinct steps planned after merging
 * identical ones, of launches per call, and of operands that the plan's
 * packed-FP32 and tensor-core steps gather into a packed workspace per call
 * (an intermediate laid out as a dense K x rows matrix for a packed-FP32
 * step is read in place and not counted), and the device bytes the plan
 * keeps between calls (intermediate arena, offset tables, descriptors,
 * split-K partials, packed-operand workspace).  Any output may be NULL.
 * INVALID_ARG if not planned yet. */
rosnet_status rosnet_plan_stats(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                const rosnet_opts *opts, void *stream, int64_t *steps_requested,
                                int64_t *steps_planned, int64_t *launches, int64_t *packed_operands,
                                int64_t *device_bytes);

/* Spill the cached plan of these arguments (as rosnet_plan_stats) to pinned
 * host memory, the out-of-core tier applied to a plan (Sec. I and III): once
 * the work enqueued on `stream` and the plan's own work have finished (the
 * call waits for them), its offset tables are copied to page-locked host
 * memory and all its device memory (tables, descriptors, intermediate arena,
 * split-K and packed-operand workspaces) and its captured graph are released;
 * rosnet_plan_stats then reports 0 device bytes.  The next contraction with
 * the same arguments restores it -- the buffers allocated again, the tables
 * copied back, the graph captured again -- instead of planning anew, with
 * the same results.  *host_bytes (may be NULL) receives the page-locked bytes
 * held while spilled.  Spilling a spilled plan does nothing.  INVALID_ARG if
 * no such plan is cached. */
rosnet_status rosnet_plan_spill(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                const rosnet_opts *opts, void *stream, int64_t *host_bytes);

/* Free the cached plan of these arguments (as rosnet_plan_stats), e.g. for a
 * server that bounds the device memory its resident plans hold.  Work the
 * plan already enqueued completes normally (buffers are released in stream
 * order); a later call with the same arguments plans again.  INVALID_ARG if
 * no such plan is cached. */
rosnet_status rosnet_plan_release(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                  const rosnet_opts *opts, void *stream);

/*
 * out = sum of the n tensors ts[0..n) in FP64, in that order (deterministic):
 * e.g. the sum over slices of a sliced network's results (Sec. II-B).  The
 * summands must share dtype, shape and block shape and be dense block-major
 * tensors (results of tensordot/contract are); *out is a new complex128
 * tensor of that shape.  Errors: INVALID_ARG, DTYPE, SHAPE, UNSUPPORTED.
 */
rosnet_status rosnet_sum(int32_t n, const rosnet_btensor *ts, void *stream, rosnet_btensor *out);

/*
 * *out = sum over all elements x of t of |x|^2, accumulated in FP64 on the
 * GPU in a fixed order (reproducible on a given device): the normalisation
 * check of a state or of a batch of amplitudes (sum over all bitstrings of
 * |<x|C|0>|^2 = 1, Sec. II-A).  Works on views.  Enqueued on `stream` and
 * waited for (synchronous).  INVALID_ARG for NULL arguments.
 */
rosnet_status rosnet_norm2(rosnet_btensor t, void *stream, double *out);

/* ----------------------------------------------------------------------- */
/* misc                                                                     */
/* ----------------------------------------------------------------------- */
/* Wait for `stream`; returns CUDA if a kernel failed, TIMEOUT if a bounded
 * device wait of the library gave up. */
rosnet_status rosnet_sync(void *stream);

/* Launch a kernel that waits on a barrier nothing will complete, giving up
 * after budget_cycles (<= 4e9) SM cycles: the next rosnet_sync on `stream`
 * reports ROSNET_ERR_TIMEOUT.  For testing the bounded-wait path of the
 * library's kernels (no fault, no hang).  The paper has no counterpart. */
rosnet_status rosnet_selftest_timeout(int64_t budget_cycles, void *stream);

/* Measure a peak arithmetic rate of the current GPU with a microkernel, so
 * that the contraction kernels' roofline fractions can be stated against
 * measured rates (the paper has no counterpart; its block products ran on
 * CPU cores, Sec. V):
 *   ROSNET_PROBE_FFMA  FP32 fused multiply-adds on the CUDA cores
 *   ROSNET_PROBE_DFMA  FP64 fused multiply-adds on the CUDA cores
 *   ROSNET_PROBE_TF32  tcgen05.mma kind::tf32 (128 x 256 x 8), TMEM accumulators
 *   ROSNET_PROBE_BF16  tcgen05.mma kind::f16, bf16 operands (128 x 256 x 16)
 * The probe is launched once to warm up and once timed with CUDA events on
 * `stream`; *flops receives the floating-point operations of the timed launch
 * (2 per multiply-add) and *ms its device time.  Synchronous.  INVALID_ARG
 * for an unknown kind or NULL outputs; TIMEOUT if the MMA probe's bounded
 * wait gave up. */
#define ROSNET_PROBE_FFMA 0
#define ROSNET_PROBE_DFMA 1
#define ROSNET_PROBE_TF32 2
#define ROSNET_PROBE_BF16 3
rosnet_status rosnet_probe_peak(int32_t kind, void *stream, double *flops, double *ms);

/* Static, human-readable description of a status code. */
const char *rosnet_status_string(rosnet_status s);

/* Message of the last error raised on the calling thread (static storage
 * owned by the library; valid until the thread's next failing call). */
const char *rosnet_last_error(void);

/* Number of kernels the library has launched in this process (for
 * accounting; graph replays count each kernel node). */
int64_t rosnet_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* ROSNET_H */
