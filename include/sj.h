/*
 * sj.h -- C ABI of the GB300 grid-indexed Euclidean epsilon self-join.
 *
 * The operation (Gowanlock & Karsin, "GPU Accelerated Self-join for the
 * Distance Similarity Metric", Section III): given |D| points of n
 * dimensions and a distance epsilon, return every ordered pair (i, j) of point
 * ids with dist(p_i, p_j) <= epsilon, Euclidean distance.  Point ids are the
 * 0-based row numbers of the input.  Self-pairs (i, i) are included, and
 * (i, j) is returned exactly when (j, i) is.
 *
 * Membership is decided bit-exactly in FP64 as
 *     s = 0; for j = 0..n-1 { t = x_i[j] - x_j[j]; s = s + t * t; }
 *     member  <=>  s <= fl(eps * eps)
 * with every subtraction, product and sum rounded to nearest on its own (no
 * fused multiply-add).  Comparing squared values is the library's reading of
 * the Section III predicate dist <= eps; it differs from rounding sqrt(s)
 * only at rounding ties.  Both precision modes return this exact set:
 *   SJ_PREC_FP64          distances in FP64 only (the paper's arithmetic);
 *   SJ_PREC_FP32_RECHECK  distances filtered in FP32 with a proven error
 *                         margin, and only pairs within that margin of
 *                         epsilon recomputed in FP64.
 *
 * Method: the grid index of Section IV-B/C (cells of side ~epsilon, only
 * non-empty cells stored: lookup array B of sorted linear cell ids, cell
 * ranges G into the point permutation A, per-dimension masks M_j), the
 * bounded adjacent-cell search of Section IV-D, the UNICOMP duplicate-search
 * removal of Section V-B (each adjacent cell pair compared once, both ordered
 * pairs emitted), and the result batching of Section V-A (at least 3 batches
 * for host output, device result buffers bounded by a byte cap).
 *
 * Conventions for every call:
 *   - `pts` is n x d row-major FP64.  It may be a host or a device pointer;
 *     the library detects which.  The caller keeps ownership and must not
 *     change the array until the call returns (nor from a callback the
 *     call makes): calls that build an index only for themselves read
 *     device points in place, without a copy.  The library does not hold
 *     the pointer after the call returns (sj_build_index and sj_submit copy
 *     the points before they return).
 *   - A pair is two consecutive uint32 values (i, j).  Results returned in
 *     sj_result are library-owned host memory, valid until sj_result_free.
 *   - Pair order is unspecified unless sj_config.sorted = 1, which orders
 *     pairs ascending by the 64-bit key (i << 32) | j.
 *   - Points have d in [1, 16] dimensions.  For d > 8 the grid covers the
 *     six dimensions with the most cells and the search refines on all d
 *     (the 3^d search of Section IV-D degenerates beyond the paper's 2-6
 *     dimensions); the two-set join, sj_selfjoin_multi, sj_submit,
 *     sj_selfjoin_noalloc, sj_selfjoin_bruteforce_device and the margin
 *     calls of the main path take d in [1, 8].
 *   - Errors: SJ_EINVAL for a NULL argument, n = 0, d outside [1, 16],
 *     eps <= 0 or non-finite, or any NaN/Inf coordinate; SJ_ERANGE when
 *     n >= 2^32 or a dimension would need 2^31 or more cells (grids whose
 *     cell count reaches 2^63 are ordered by coordinate tuple, see
 *     sj_lookup); SJ_ENOMEM when device or pinned memory
 *     runs out; SJ_ECUDA for any other CUDA error (the message is in
 *     sj_last_error); SJ_ETIMEOUT when a bounded device wait expired;
 *     SJ_EOVERFLOW when a caller-provided output buffer is too small (the
 *     required count is still reported).
 *   - One context serves one CUDA device.  sj_submit and sj_poll may be
 *     called from any thread; all other calls on one context must not run
 *     concurrently with each other.
 */
#ifndef SJ_H
#define SJ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SJ_API __attribute__((visibility("default")))
#else
#define SJ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sj_ctx sj_ctx;
typedef struct sj_index sj_index;
typedef struct sj_result sj_result;

typedef enum {
    SJ_OK = 0,
    SJ_PENDING = 1,
    SJ_EINVAL = -1,
    SJ_ENOMEM = -2,
    SJ_ERANGE = -3,
    SJ_ECUDA = -4,
    SJ_ETIMEOUT = -5,
    SJ_EBUSY = -6,
    SJ_EOVERFLOW = -7,
    SJ_ENOTFOUND = -8
} sj_status;

typedef enum { SJ_PREC_FP64 = 0, SJ_PREC_FP32_RECHECK = 1 } sj_precision;

/* Cell lookup used by the adjacent-cell search (Section IV-D).
 * SJ_LOOKUP_SEARCH binary-searches the sorted array B of non-empty cell ids,
 * as the paper does.  SJ_LOOKUP_DENSE adds a table over all cells of the grid
 * (4 bytes per cell) that answers a lookup with one load; SJ_LOOKUP_AUTO uses
 * it when the grid has at most max(2^25, 16 n) cells.  SJ_LOOKUP_COORDS
 * orders the cells by their coordinate tuples (c_n, ..., c_1) instead of
 * linear ids (the same order, built with one radix sort per group of
 * dimensions) and binary-searches the tuples; no B is built.  It is taken
 * automatically when the grid has 2^63 or more cells, where linear ids do
 * not fit in 64 bits.  Results are identical in every mode. */
typedef enum {
    SJ_LOOKUP_AUTO = 0,
    SJ_LOOKUP_DENSE = 1,
    SJ_LOOKUP_SEARCH = 2,
    SJ_LOOKUP_COORDS = 3
} sj_lookup;

/* Coordinate frame of the FP32 point records of SJ_PREC_FP32_RECHECK.
 * SJ_FRAME_GRID stores fl32(x_j - g_min_j): its rounding error grows with
 * the extent of the data, so the margin of values recomputed in FP64 widens
 * with range / eps and the filter is dropped (FP64 arithmetic) beyond about
 * 2e6.  SJ_FRAME_CELL stores each coordinate relative to a frame that
 * repeats every four cells (the kernel undoes the frame step exactly), so
 * the error is a few units in the last place of the cell side at any
 * range.  SJ_FRAME_AUTO (default) keeps the grid frame while its margin is
 * below 2^-10 eps^2, else takes the narrower margin.  Results are
 * identical in every frame. */
typedef enum { SJ_FRAME_AUTO = -1, SJ_FRAME_GRID = 0, SJ_FRAME_CELL = 1 } sj_frame;

typedef struct {
    int32_t prec;            /* sj_precision; default SJ_PREC_FP32_RECHECK */
    int32_t unicomp;         /* 1 (default): Section V-B duplicate-search removal;
                                0: every point searches all 3^n adjacent cells
                                (Algorithm 1) and emits only (p, q) */
    uint64_t out_cap_bytes;  /* device memory for result batches of calls that
                                return host results; default 2 GiB */
    int32_t min_batches;     /* minimum result batches for host results
                                (Section V-A uses 3); default 3 */
    int32_t sorted;          /* 1: host results sorted by (i << 32) | j */
    int32_t autotune;        /* 1 (default): the launch parameters of a
                                single join's search-and-refine launch
                                (grab, chunk ring depth, pair staging size,
                                item slots, warps per block) come from the
                                tuner, which times sampled count-only
                                launches the first time a (d, precision,
                                UNICOMP, points-per-cell bucket) key is met
                                in the process and reuses the choice after;
                                the many-join launch of sj_selfjoin_multi
                                and sj_submit takes the wave tuner's choice
                                (grab, ring depth, staging size, item
                                slots for every job of a wave), which times
                                the multi-join launch of the first wave of
                                a (precision, log2 points per SM) key of at
                                least 2^17 points with each candidate and
                                reuses the choice after; 0: fixed defaults.
                                Never changes the result. */
    int32_t device;          /* CUDA device ordinal; default 0 */
    int32_t lookup;          /* sj_lookup; default SJ_LOOKUP_AUTO */
    int32_t profile;         /* 1: time every join-kernel launch with CUDA
                                events (read with sj_profile_read) */
    int32_t max_inflight;    /* sj_submit: most requests admitted at once; default 64 */
    uint64_t serve_mem_bytes;/* sj_submit: device bytes the admitted requests may
                                hold together; default 8 GiB */
    /* launch tuning of the search-and-refine kernel; -1 (default) lets the
     * library (or the tuner, with autotune = 1) choose */
    int32_t grab;            /* work items a warp takes per cursor bump */
    int32_t nbuf;            /* candidate-chunk ring depth (2..8) */
    int32_t staging;         /* staged pairs per warp (128, 256, 512 or 1024) */
    int32_t wpb;             /* warps per block (1, 2, 4 or 8) */
    int32_t slots;           /* work items a warp holds at once (1 or 2) */
    int32_t frame;           /* sj_frame; default SJ_FRAME_AUTO */
    int32_t wait_ms;         /* limit of every bounded wait inside the search
                                kernel (a warp waiting for its staged
                                candidate copies), in ms; 0 (default): 2000.
                                A wait that expires ends the call with
                                SJ_ETIMEOUT and leaves the context usable. */
    int32_t test_stall;      /* test hook, 0 (default) in normal use.  1: in
                                every single-join search launch of this
                                context, warp 0 of block 0 never issues its
                                first candidate copy, so its wait for that
                                copy expires after wait_ms (no copy is in
                                flight for it) and the call returns
                                SJ_ETIMEOUT.  Lets a test drive the time-out
                                path without any fault. */
} sj_config;

/* Fills *cfg with the defaults listed above. */
SJ_API void sj_config_default(sj_config *cfg);

/* Creates a context on cfg->device (NULL cfg: defaults).  *out is set on
 * success.  Errors: SJ_EINVAL, SJ_ECUDA (no such device), SJ_ENOMEM. */
SJ_API sj_status sj_create(const sj_config *cfg, sj_ctx **out);

/* Destroys the context.  Results and indexes it produced stay valid;
 * pending sj_submit requests are cancelled.  NULL is ignored. */
SJ_API void sj_destroy(sj_ctx *ctx);

/* Message of the last error on this context ("" if none); valid until the
 * next call on the context. */
SJ_API const char *sj_last_error(const sj_ctx *ctx);

/* Static name of a status code. */
SJ_API const char *sj_status_str(sj_status st);

/* ------------------------------------------------------------------ */
/* Grid index (Section IV-B, IV-C).                                   */
/* ------------------------------------------------------------------ */

/* Builds the grid index of pts on the device: bounds g_min = min - eps and
 * g_max = max + eps per dimension (Section IV-B), cells of side
 * w = eps * (1 + 2^-16), |g_j| = floor((g_max_j - g_min_j) / w) + 1 cells in
 * dimension j, linear cell ids with dimension 1 fastest, the arrays B, G, A
 * and M_j of Section IV-C, and the cell-ordered coordinate copies the
 * search reads.  The index owns device memory until sj_index_free; pts is
 * not referenced after the call.  Errors as listed in the file comment. */
SJ_API sj_status sj_build_index(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                         double eps, sj_index **out);

/* Frees the index and its device memory.  NULL is ignored. */
SJ_API void sj_index_free(sj_index *idx);

/* Sizes and geometry of an index. */
typedef struct {
    uint64_t n;              /* |D| */
    int32_t d;               /* n in the paper's notation: dimensions */
    int32_t dense;           /* 1 when the dense lookup table was built */
    double eps;
    double cell_width;       /* w */
    uint64_t n_cells;        /* |G| = |B|, non-empty cells */
    uint64_t grid_cells;     /* product of |g_j|, all cells of the grid
                                (2^64 - 1 when it reaches 2^63) */
    double gmin[8], gmax[8]; /* g_min_j, g_max_j */
    int64_t ng[8];           /* |g_j| */
    uint64_t device_bytes;   /* device memory the index holds */
    int32_t fp32;            /* 1: the FP32 filter has a usable margin on this grid */
    int32_t frame;           /* sj_frame of the index's FP32 records */
    int32_t grid_d;          /* dimensions the grid covers: d, or 6 when d > 8 */
    int32_t grid_dim[8];     /* the point dimension of each grid dimension; eps,
                                gmin, gmax, ng, n_cells, grid_cells and the
                                arrays of sj_index_export describe these */
} sj_index_desc;

SJ_API sj_status sj_index_info(const sj_index *idx, sj_index_desc *out);

/* Copies the Section IV-C arrays to host memory (any pointer may be NULL):
 *   B[n_cells]          sorted linear ids of the non-empty cells (not
 *                       built for cells ordered by coordinate tuple:
 *                       a non-NULL B then gives SJ_ERANGE);
 *   G[n_cells + 1]      cell h holds A[G[h] .. G[h+1]);
 *   A[n]                point ids in cell order;
 *   M[d * ceil(max_j |g_j| / 32)]  bit c of row j is set when some point
 *                       has cell coordinate c in dimension j.
 * For tests and tools; synchronous. */
SJ_API sj_status sj_index_export(const sj_index *idx, uint64_t *B, uint32_t *G,
                          uint32_t *A, uint32_t *M);

/* The classification margin of SJ_PREC_FP32_RECHECK for a grid with
 * dimension d, distance eps and padded bounds g_min_j, g_max_j
 * (Section IV-B: g_min_j = min_j - eps, g_max_j = max_j + eps), with FP32
 * records relative to g_min (SJ_FRAME_GRID).  The join kernel computes an
 * FP32 squared distance s32 from coordinates relative to the centre of the
 * query's cell (see the derivation in csrc/margin.cu); s32 <= *lo implies
 * membership by the exact FP64 test, s32 > *hi implies non-membership, and
 * only values in between are recomputed in FP64.  *w32 receives the cell
 * side rounded to FP32.  Host-only, no device needed.  Returns SJ_ERANGE
 * when this frame has no useful margin (the FP32 mode then takes the cell
 * frame, see sj_frame, or computes in FP64), SJ_EINVAL for bad arguments. */
SJ_API sj_status sj_fp32_margin(int d, double eps, const double *gmin, const double *gmax,
                                float *w32, float *lo, float *hi);

/* The same margin for the records of frame `frame` (SJ_FRAME_GRID, the
 * frame of sj_fp32_margin, or SJ_FRAME_CELL; see sj_frame).  In the cell
 * frame a record holds fl32(fl64(fl64(x_j - g_min_j) - fl64(4 K_j w))) with
 * K_j = floor(c_j / 4) for the point's cell c_j, and the kernel moves a
 * candidate of the neighbouring frame by 4 * w32 (derivation in
 * csrc/margin.cu).  Errors as sj_fp32_margin, SJ_EINVAL for another frame. */
SJ_API sj_status sj_fp32_margin_frame(int d, double eps, const double *gmin,
                                      const double *gmax, int frame, float *w32, float *lo,
                                      float *hi);

/* The margin of the FP32 filter for points of more than 8 dimensions
 * (d <= 16) in the expanded form: the grid frame's sum |z_p|^2 + |z_q|^2
 * - 2 z_p . z_q over all d dimensions, z_j = fl32(y_j - o_j), with the
 * origin o_j at the home cell centre in a grid dimension (grid[j] != 0;
 * the search covers the home cell's neighbours there) and at *mid[j] =
 * fl32((fmax_j - fmin_j) / 2) in the others (written for j < d; 0 for grid
 * dimensions).  y_j = fl32(fl64(x_j - fmin_j)), fmin_j = min_j - eps,
 * fmax_j = max_j + eps (derivation in csrc/margin.cu).  s32 <= *lo implies
 * membership, s32 > *hi non-membership.  Returns SJ_ERANGE when no useful
 * margin exists (the search then takes the difference form below),
 * SJ_EINVAL for bad arguments.  Host-only. */
SJ_API sj_status sj_fp32_margin_hd(int d, double eps, const double *fmin, const double *fmax,
                                   const int *grid, float *lo, float *hi, float *mid);

/* The margin of the FP32 filter for points of more than 8 dimensions
 * (d <= 16) in the difference form, used where the expanded form has no
 * useful margin: the search sums fl32(y_p,j - y_q,j)^2 with fused
 * multiply-adds over all d dimensions, y_j = fl32(fl64(x_j - fmin_j)),
 * fmin_j = min_j - eps, fmax_j = max_j + eps (derivation in
 * csrc/margin.cu).  s32 <= *lo implies membership, s32 > *hi
 * non-membership.  Returns SJ_ERANGE when no useful margin exists (those
 * joins then compute in FP64), SJ_EINVAL for bad arguments.  Host-only. */
SJ_API sj_status sj_fp32_margin_diff(int d, double eps, const double *fmin,
                                     const double *fmax, float *lo, float *hi);

/* Measured FP32 rate of this GPU, the denominator of the search kernel's
 * roofline (the paper has no counterpart; it measures on other hardware).
 * Runs independent FP32 fused multiply-add chains on every SM of `device`
 * at full occupancy, scalar fma.rn.f32 (packed = 0) or packed
 * fma.rn.f32x2 (packed = 1), and reports the best of five timed launches:
 * *tflops counts two FLOPs per FMA lane, *ms is that launch's time.
 * Allocates a small device buffer (one float per thread) and a stream for
 * the call.  Errors: SJ_EINVAL for NULL outputs or a negative device,
 * SJ_ECUDA when the device or a launch fails. */
SJ_API sj_status sj_fp32_fma_rate(int device, int packed, double *tflops, double *ms);

/* Measured FP64 rate of this GPU, the denominator of the plain FP64 join's
 * roofline (the paper has no counterpart).  Independent fma.rn.f64 chains
 * on every SM of `device` at full occupancy, the best of five timed
 * launches: *tflops counts two FLOPs per FMA, *ms is that launch's time.
 * Allocates a small device buffer and a stream for the call.  Errors as
 * sj_fp32_fma_rate. */
SJ_API sj_status sj_fp64_fma_rate(int device, double *tflops, double *ms);

/* ------------------------------------------------------------------ */
/* Self-join.                                                         */
/* ------------------------------------------------------------------ */

/* The full join into library-owned host memory: builds the index, sizes the
 * result from a sampled count pass, and streams the pairs out in
 * max(min_batches, needed) batches whose device buffers stay within
 * out_cap_bytes, overlapping each batch's kernel with the previous batch's
 * copy to the host (Section V-A).  A batch that overflows its buffer is
 * split and re-run.  *out is set on success. */
SJ_API sj_status sj_selfjoin(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                      double eps, sj_result **out);

/* The same on a built index (which is not modified). */
SJ_API sj_status sj_selfjoin_index(sj_ctx *ctx, const sj_index *idx, sj_result **out);

/* Device-resident join: d_pairs is a device buffer of cap_pairs pairs
 * (2 * cap_pairs uint32).  All work is enqueued on `stream` (a cudaStream_t;
 * NULL = the legacy default stream) and the call returns once *count is
 * known.  *count receives the number of pairs even when it exceeds
 * cap_pairs; then only the first cap_pairs are written and the call returns
 * SJ_EOVERFLOW.  pts may be host or device memory. */
SJ_API sj_status sj_selfjoin_device(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                             double eps, uint32_t *d_pairs, uint64_t cap_pairs,
                             uint64_t *count, void *stream);

/* Device-resident join on a built index. */
SJ_API sj_status sj_selfjoin_index_device(sj_ctx *ctx, const sj_index *idx,
                                   uint32_t *d_pairs, uint64_t cap_pairs,
                                   uint64_t *count, void *stream);

/* Two-set join R ⋈ S (the paper treats the self-join as a special case of
 * this join): all pairs (i, j) with point i of R and point j of S within
 * eps, by the same predicate as the self-join.  One grid (Section IV-B) is
 * laid over the bounding box of R ∪ S; S is indexed as the candidate set
 * and the points of R are the queries, grouped by their cells; every query
 * cell searches all 3^n adjacent cells (UNICOMP does not apply: the pair
 * (i, j) has one orientation).  A pair is (index in R, index in S).  R and S
 * may be host or device memory.  Output, count and errors as
 * sj_selfjoin_device. */
SJ_API sj_status sj_join2_device(sj_ctx *ctx, const double *R, uint64_t nR, const double *S,
                                 uint64_t nS, int d, double eps, uint32_t *d_pairs,
                                 uint64_t cap_pairs, uint64_t *count, void *stream);

/* The index-free comparator: every ordered pair (i, j) is tested with the
 * exact FP64 predicate (no grid, no UNICOMP, no FP32 filter), O(n^2)
 * evaluations.  It returns the same pair set as sj_selfjoin_device and
 * exists to measure what the grid index of Section IV and the
 * duplicate-search removal of Section V-B save (the paper compares its
 * indexed GPU join with a brute-force GPU join).  Arguments, output and
 * errors as sj_selfjoin_device. */
SJ_API sj_status sj_selfjoin_bruteforce_device(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                                               double eps, uint32_t *d_pairs, uint64_t cap_pairs,
                                               uint64_t *count, void *stream);

/* Counts the pairs without writing them. */
SJ_API sj_status sj_selfjoin_count(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                            double eps, uint64_t *count);

/* Streaming join: like sj_selfjoin, but each batch is handed to `cb` as it
 * arrives (pairs points to 2 * k uint32 in pinned host memory, valid only
 * during the callback) instead of being gathered.  A non-zero return from cb
 * stops the join (the call then returns SJ_OK after the batches in flight
 * finish, with no more callbacks). */
typedef int (*sj_chunk_cb)(const uint32_t *pairs, uint64_t k, void *user);
SJ_API sj_status sj_selfjoin_stream(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                             double eps, sj_chunk_cb cb, void *user);

/* Join for callers that cannot allocate memory (the paper has no
 * counterpart; this is a deployment convenience).  Some callers may not call
 * cudaMalloc or any allocating routine: code running inside another
 * framework's pre-reserved memory budget, or code that must account for
 * every allocation up front.  This call runs the same index build and
 * search-and-refine kernels as sj_selfjoin_device (FP32 filter + FP64
 * recheck, UNICOMP) without a context and allocates nothing: all working
 * memory comes from one fixed region of 24 MiB that every GPU loading the
 * library holds until the process exits.
 *   d_pts    n x d row-major FP64, device memory, not modified;
 *   d_pairs  device buffer of cap_pairs pairs (2 * cap_pairs uint32);
 *   count    receives the pair count (also when it exceeds cap_pairs: then
 *            only cap_pairs pairs are written and SJ_EOVERFLOW returned);
 *   stream   a cudaStream_t (NULL: legacy default stream); the call waits
 *            for it before returning;
 *   msg      optional buffer of msg_len bytes for an error message.
 * Limits: n <= 65536 points, d in [1, 8], and at most 2^20 grid cells of
 * side ~eps over the points' bounding box, else SJ_ERANGE; host pointers
 * are rejected with
 * SJ_EINVAL.  The region's device address is looked up on the first call on
 * each device (make that first call before any stream capture).  Calls share
 * the region: they are serialised within the process, and work that
 * overlaps with them on the GPU through the same region would race. */
SJ_API sj_status sj_selfjoin_noalloc(const double *d_pts, uint64_t n, int d, double eps,
                                     uint32_t *d_pairs, uint64_t cap_pairs, uint64_t *count,
                                     void *stream, char *msg, size_t msg_len);

/* ------------------------------------------------------------------ */
/* Results.                                                           */
/* ------------------------------------------------------------------ */

SJ_API uint64_t sj_result_count(const sj_result *r);
SJ_API const uint32_t *sj_result_pairs(const sj_result *r);   /* 2 * count uint32 */
SJ_API void sj_result_free(sj_result *r);                     /* NULL is ignored */

/* ------------------------------------------------------------------ */
/* One join split over several ranks (one process per GPU).           */
/* ------------------------------------------------------------------ */

/* The share of rank `rank` of `world` in one join: the rank builds the grid
 * index of all points (Section IV-B/C, the same on every rank) and
 * searches only the query cells of its shard, emitting the pairs whose
 * home cell (under UNICOMP, the cell that visits the cell pair, Section V-B)
 * is one of them.  The ranks' outputs are disjoint and their union is the
 * full result; summing the counts (one all-reduce) is the only exchange.
 * Shards are contiguous ranges of work items (cell, block of 32 points)
 * cut at cell starts, balanced by the estimated search cost of the items
 * (see sj_shard_bounds_cost; the costs are computed on the device).
 * Arguments and errors as sj_selfjoin_device, plus SJ_EINVAL unless
 * 0 <= rank < world. */
SJ_API sj_status sj_selfjoin_shard_device(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                                          double eps, int rank, int world, uint32_t *d_pairs,
                                          uint64_t cap_pairs, uint64_t *count, void *stream);

/* The shard rule on a host array, needing no device: item_block[k] is the
 * block index within its cell of work item k (0 at a cell start; items in
 * cell order).  [*lo, *hi) is [n r / w, n (r + 1) / w) with each bound moved
 * forward to the next cell start (or n).  The ranks' ranges tile [0, n). */
SJ_API sj_status sj_shard_bounds(const uint32_t *item_block, uint64_t n_items, int rank,
                                 int world, uint64_t *lo, uint64_t *hi);

/* The cost-balanced shard rule of sj_selfjoin_shard_device on host arrays:
 * item_cost[k] is the estimated search cost of work item k (the device
 * uses K (q + 20) + 2000 with K the item's candidate points and q its query
 * points).  With C the total cost, the bound between ranks r - 1 and r is
 * the cell start whose exclusive cost prefix is nearest to C r / w (of the
 * two starts around the first item whose prefix reaches C r / w; the later
 * on a tie).  The ranks' ranges tile [0, n), and a rank's cost exceeds
 * C / w by at most the cost of one cell. */
SJ_API sj_status sj_shard_bounds_cost(const uint32_t *item_block, const uint64_t *item_cost,
                                      uint64_t n_items, int rank, int world, uint64_t *lo,
                                      uint64_t *hi);

/* ------------------------------------------------------------------ */
/* Many joins at once.                                                */
/* ------------------------------------------------------------------ */

/* One join of a multi-join call: n x d row-major FP64 points (host or device
 * memory, owned by the caller) and its epsilon. */
typedef struct {
    const double *pts;
    uint64_t n;
    int32_t d;
    int32_t pad;
    double eps;
} sj_job;

/* Runs n_jobs independent self-joins of uneven n, d and eps together
 * (Section IV and V for each job; the paper runs one join at a time).  The
 * jobs are grouped into waves of at most 64 whose estimated device memory
 * fits in serve_mem_bytes; per wave the points of all jobs are bounded in
 * one launch (one host read-back), then one replay of a captured CUDA graph
 * builds every job's grid index with batched kernels (each launch covers
 * all jobs of the wave) and runs ONE persistent search-and-refine launch in
 * which every warp works through all jobs' work items.  Jobs whose grid is
 * too large for the dense cell table run alone through sj_selfjoin.
 * out[i] receives job i's result (library-owned host memory, free with
 * sj_result_free; pair order unspecified unless sorted = 1) and, when
 * status is not NULL, status[i] its status.  Returns SJ_OK when every job
 * succeeded, else the first job error (message in sj_last_error); the other
 * jobs' results are still returned.  sj_last_stats sums over the jobs
 * (batches = waves, retries = jobs re-joined alone because their result
 * outgrew its estimated buffer); its grab, nbuf and staging are the last
 * wave's launch parameters and tuned is 2 when a wave of the call was
 * tuned, 1 when a wave took the wave tuner's cached choice, else 0. */
SJ_API sj_status sj_selfjoin_multi(sj_ctx *ctx, const sj_job *jobs, uint64_t n_jobs,
                                   sj_result **out, sj_status *status);

/* ------------------------------------------------------------------ */
/* Statistics of the last join on a context.                          */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t pairs;          /* pairs returned */
    uint64_t evaluations;    /* point-pair distance evaluations the method
                                requires: sum over visited cell pairs of
                                |C_a| |C_b|, home cells |C| (|C| - 1) / 2 under
                                UNICOMP (|C|^2 without) */
    uint64_t rechecks;       /* FP32 results inside the margin, recomputed in FP64 */
    uint64_t n_cells;        /* |G| */
    uint32_t batches;        /* result batches */
    uint32_t retries;        /* batches re-run after an overflow */
    uint64_t estimate;       /* pair count predicted by the sampled pass */
    double ms_index;         /* host wall time of the index build */
    double ms_join;          /* host wall time of the join after the index */
    double ms_total;
    uint64_t kernel_launches;/* CUDA kernels the library launched for the call */
    /* launch parameters of the search-and-refine kernel for the call */
    int32_t grab;            /* work items per cursor bump */
    int32_t nbuf;            /* candidate-chunk ring depth (0: by dimension) */
    int32_t wpb;             /* warps per block (0: by occupancy) */
    int32_t tuned;           /* 0 defaults, 1 from the tuner's cache, 2 tuned by this call */
    int32_t staging;         /* staged pairs per warp (0: by dimension) */
    int32_t frame;           /* sj_frame of the FP32 filter used by the call;
                                -1 when every distance was computed in FP64 */
} sj_stats;

SJ_API sj_status sj_last_stats(const sj_ctx *ctx, sj_stats *out);

/* With sj_config.profile = 1: total device time (ms, CUDA events on the
 * launching stream) and launch count of the search-and-refine kernel since
 * the last read; resets both.  Synchronises the context's work. */
SJ_API sj_status sj_profile_read(sj_ctx *ctx, double *kernel_ms, uint64_t *launches);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of join requests.                     */
/* ------------------------------------------------------------------ */

/* Queues a self-join request and returns at once with a ticket.  The pts
 * buffer is copied before sj_submit returns.  A scheduler thread admits
 * queued requests while fewer than max_inflight are running and their
 * estimated device memory fits in serve_mem_bytes; admitted requests share
 * persistent multi-join kernel launches, so requests that arrive while
 * others run overlap with them on the device.  Errors: as sj_selfjoin for
 * the arguments, SJ_ENOMEM if the request alone exceeds serve_mem_bytes;
 * a NaN or infinite coordinate is reported by sj_poll (SJ_EINVAL). */
SJ_API sj_status sj_submit(sj_ctx *ctx, const double *pts, uint64_t n, int d,
                    double eps, uint64_t *ticket);

/* SJ_PENDING while the request runs; SJ_OK with *out set when it finished
 * (the ticket is then consumed); the request's error otherwise;
 * SJ_ENOTFOUND for an unknown ticket.  wait_ms > 0 blocks up to that long. */
SJ_API sj_status sj_poll(sj_ctx *ctx, uint64_t ticket, int wait_ms, sj_result **out);

/* Counters of the serving scheduler of a context (all zero before the first
 * sj_submit). */
typedef struct {
    uint64_t submitted, completed;
    uint64_t waves;            /* multi-join waves run */
    uint64_t max_wave;         /* most requests in one wave */
    uint64_t overflow_reruns;  /* requests re-joined after their estimate was short */
    uint64_t standalone;       /* requests run through the stand-alone path */
    uint64_t graph_launches;   /* CUDA graph replays */
    uint64_t queued;           /* waiting for admission now */
    uint64_t mem_in_use;       /* estimated device bytes admitted now */
    int32_t inflight;          /* admitted requests now */
    int32_t lanes;             /* waves that may run at the same time */
    int32_t max_concurrent_waves; /* most waves seen running at once */
    int32_t reserved;
    /* host wall time summed over the lanes' waves (ms): points to the device
     * and the bounds pass, the graph replay (index build + join), the result
     * copies to the host */
    double ms_bounds, ms_graph, ms_output;
    uint64_t tuned_waves;      /* waves whose multi-join launch the wave tuner timed */
    double ms_tune;            /* host wall time of those tuning passes (ms) */
} sj_serve_info;

SJ_API sj_status sj_serve_stats(sj_ctx *ctx, sj_serve_info *out);

/* Forgets every choice of the launch tuners of the process (single joins
 * and many-join waves), so that the next join or wave of each key is tuned
 * again.  Safe while no join is running. */
SJ_API void sj_tune_reset(void);

/* Per-request timestamps (seconds since the context was created) of a
 * finished result: submitted, admitted, completed.  Zero for results not
 * produced by sj_submit. */
SJ_API sj_status sj_result_times(const sj_result *r, double *t_submit, double *t_admit,
                          double *t_done);

#ifdef __cplusplus
}
#endif

#endif /* SJ_H */
