// sj_internal.cuh -- internal declarations of the GB300 self-join library.
//
// Layout of the library:
//   scan.cu      device-wide exclusive scan (u32) used by the index build
//   sort.cu      LSD radix sort of (u64 key, u32 value) for grids too large
//                for the dense cell table
//   index.cu     grid index build (Section IV-B, IV-C): bounds, cell ids,
//                counting, radix or coordinate-tuple sort by cell, B / G / A /
//                M_j, cell-ordered FP32 and FP64 point records, work items;
//                the projected grid of points with more than 8 dimensions
//   margin.cu    the proven FP32 filter margins (grid frame, cell frame,
//                difference form)
//   join_dev.cuh device helpers shared by the search kernels (row templates,
//                candidate ranges, packed FP32 pairs)
//   join.cu      the persistent search-and-refine kernel (Section IV-D, IV-E,
//                V-B) in both precision modes, and its launches
//   hd_join.cu   the search kernel for 9 to 16 dimensions
//   brute.cu     the index-free comparator
//   engine.cu    many joins in one persistent launch, replayed as a CUDA graph
//   serve.cu     the serving loop (continuous batching of join requests)
//   tune.cu      the launch tuner
//   shard.cu     one join split over ranks
//   noalloc.cu   the join without allocation
//   api.cu       the C ABI of include/sj.h: contexts, batching (Section V-A),
//                results, statistics
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/sj.h"

namespace sj {

constexpr int kMaxDim = 8;             // grid dimensions, and point dimensions of the main path
constexpr int kMaxPointDim = 16;       // point dimensions (d > kMaxDim: high-dimensional path)
constexpr int kHdGridDims = 6;         // grid dimensions of the high-dimensional path
constexpr int kWarpsPerBlock = 8;      // 256 threads per block, as in Section VI-B
constexpr int kQueryBlock = 32;        // query points per work item
constexpr uint32_t kErrTimeout = 1u;   // device error word bits
constexpr uint32_t kErrBadRange = 2u;

// Status propagation ---------------------------------------------------------

struct Error {
    sj_status st = SJ_OK;
    std::string msg;
};

#define SJ_CUDA_TRY(expr)                                                        \
    do {                                                                         \
        cudaError_t e__ = (expr);                                                \
        if (e__ != cudaSuccess) {                                                \
            ::sj::set_cuda_error(err, e__, #expr, __FILE__, __LINE__);           \
            return err.st;                                                       \
        }                                                                        \
    } while (0)

#define SJ_TRY(expr)                                                             \
    do {                                                                         \
        sj_status s__ = (expr);                                                  \
        if (s__ != SJ_OK) return s__;                                            \
    } while (0)

void set_cuda_error(Error &err, cudaError_t e, const char *expr, const char *file, int line);
sj_status fail(Error &err, sj_status st, const std::string &msg);

// Device memory from the stream-ordered pool of the context's device.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
sj_status dev_alloc(Error &err, DevBuf &b, size_t bytes, cudaStream_t s);
void dev_free(DevBuf &b, cudaStream_t s);

// Grid geometry (Section IV-B), computed on the host from the bounds.
struct Geometry {
    int d = 0;
    uint64_t n = 0;
    double eps = 0, E2 = 0, w = 0;
    double gmin[kMaxDim] = {}, gmax[kMaxDim] = {};
    int64_t ng[kMaxDim] = {};
    uint64_t stride[kMaxDim] = {};     // linear id = sum c_j * stride[j], stride[0] = 1
    uint64_t grid_cells = 0;           // product of ng (saturated when huge)
    // 1: the grid has 2^63 or more cells, so linear ids do not fit in 64
    // bits; cells are then ordered and searched by coordinate tuple
    int huge = 0;
    // FP32 filter thresholds: s32 <= lo32 -> member, s32 > hi32 -> not a
    // member, otherwise recompute in FP64.  fp32_ok = 0 when the margin is
    // unusable and the FP32 mode falls back to FP64 arithmetic.
    float lo32 = -1.0f, hi32 = 0.0f;
    float w32 = 0.0f;                  // fl32(w): cell side in the FP32 frame
    float w4 = 0.0f, inv_w4 = 0.0f;    // 4 w32 and fl32(1 / (4 w32)): cell frame step
    int frame = 0;                     // sj_frame of the FP32 records (grid or cell)
    int fp32_ok = 0;
};

// Device-resident grid index.
struct Index {
    Geometry g;
    int dense = 0;                 // dense lookup table built
    int tuple = 0;                 // cells sorted and searched by coordinate tuple (no B)
    uint64_t n_cells = 0;          // |G|
    uint32_t n_items = 0;          // work items (cell, query block)
    uint32_t max_cell = 0;         // largest cell population
    int rs32 = 0, rs64 = 0;        // record strides (floats / doubles)
    DevBuf pts;                    // n x d FP64 input (row-major): a copy, or the caller's array
    int pts_borrowed = 0;          // pts is the caller's device array (not freed with the index)
    DevBuf rec32;                  // cell-ordered FP32 records: y_0..y_{d-1}, id
    DevBuf rec64;                  // cell-ordered FP64 records: x_0..x_{d-1}, id
    DevBuf A;                      // u32[n] point ids in cell order
    DevBuf B;                      // u64[|G|] sorted linear ids of non-empty cells
    DevBuf G;                      // u32[|G|+1] cell starts in cell order
    DevBuf cc;                     // i32[|G| * d] cell coordinates
    DevBuf M;                      // u32[d * mwords] occupancy bitmaps M_j
    DevBuf lut;                    // u32[grid_cells + 1] dense: points in cells with smaller id
    DevBuf items;                  // uint2[n_items] (cell h, query block)
    DevBuf counts_dev;             // device counters: bounds, |G|, work items
    uint32_t mwords = 0;
    int counts_read = 0;
    // build counters copied to pinned host memory mid-build (BuildOpts):
    // valid once early_ev has completed; [1] = |G|
    const uint32_t *early_counts = nullptr;
    cudaEvent_t early_ev = nullptr;
    uint64_t bytes = 0;
    cudaStream_t owner_stream = nullptr;
    // Points of more than kMaxDim dimensions: the grid (g, and every array
    // above) covers the kHdGridDims dimensions gdim[] with the most cells,
    // built from the projected points; the search refines on all dfull
    // coordinates, read from the cell-ordered records below.  g.lo32, g.hi32
    // and g.fp32_ok then hold the margin of the difference-form FP32 sum
    // (margin.cu, fp32_margin_diff).
    int dfull = 0;                 // point dimensions (g.d when dfull <= kMaxDim)
    int gdim[kMaxDim] = {};        // original dimension of grid dimension j
    double fmin[kMaxPointDim] = {}, fmax[kMaxPointDim] = {};  // min - eps, max + eps, all dims
    DevBuf ptsd;                   // n x dfull FP64 input (row-major), exact rechecks
    DevBuf recd32;                 // cell-ordered fl32(x_j - fmin_j), j < dfull, then the id
    DevBuf recd64;                 // cell-ordered x_j, j < dfull, then the id
    int rsd32 = 0, rsd64 = 0;      // their strides (floats / doubles)
    // FP32 sum of the search: expanded form (origin mid32[j] outside the grid
    // dimensions) when its margin is usable, else the difference form
    int hd_exp = 0;
    float hmid[kMaxPointDim] = {};
    DevBuf hmid_dev;               // hmid in device memory
};

// FP32 margin of the expanded-form sum of the high-dimensional kernel
// (margin.cu): grid[j] != 0 marks the grid dimensions (origin at the home
// cell centre), the others take their origin mid32[j] = fl32(X_j / 2).
// Returns false when no useful margin exists.
bool fp32_margin_hd(int d, double eps, const double *fmin, const double *fmax, const int *grid,
                    float *lo32, float *hi32, float *mid32);
// FP32 margin of the high-dimensional path (margin.cu): the kernel sums
// fl32(y_p - y_q)^2 with fused multiply-adds over all d dimensions,
// y = fl32(fl64(x_j - fmin_j)).  Returns false when no useful margin exists.
bool fp32_margin_diff(int d, double eps, const double *fmin, const double *fmax, float *lo32,
                      float *hi32);
// FP32 filter margin of a geometry (margin.cu): chooses the record frame
// (frame_mode: an sj_frame) and sets frame, w32, w4, inv_w4, lo32, hi32 and
// fp32_ok.
void fp32_margin(Geometry &g, int frame_mode);

// Options of build_index.
struct BuildOpts {
    // when the points are device memory of the current device, the index
    // reads them in place instead of copying them; only for indexes freed
    // before the caller's array may change (within one synchronous call)
    bool borrow_pts = false;
    // when set: the build counters (4 uint32, [1] = |G|) are copied to this
    // pinned host memory as soon as |G| is known and ev_counts is recorded
    // after the copy, so that the host can choose launch parameters while
    // the rest of the index builds (Index::early_counts)
    uint32_t *h_counts = nullptr;
    cudaEvent_t ev_counts = nullptr;
};

// given_mm: per-dimension bounds (order keys, min/max interleaved) of a grid
// shared with another point set; null to bound the points themselves.
// frame_mode: the sj_frame of the FP32 records (SJ_FRAME_AUTO chooses).
sj_status build_index(Error &err, const double *pts_any, uint64_t n, int d, double eps,
                      int lookup_mode, int frame_mode, cudaStream_t s, Index &ix,
                      const unsigned long long *given_mm = nullptr, const BuildOpts *opt = nullptr);
// Per-dimension min/max (order keys) of device points and a non-finite flag
// (synchronises s).
sj_status bounds_of(Error &err, const double *d_pts, uint64_t n, int d, cudaStream_t s,
                    unsigned long long *mm, bool *nonfinite);
void free_index(Index &ix, cudaStream_t s);
sj_status ensure_rec64(Error &err, Index &ix, cudaStream_t s);
// Build into a caller-provided device region, allocating nothing (index.cu).
sj_status build_index_static(Error &err, const double *d_pts, uint64_t n, int d, double eps,
                             unsigned char *region, size_t region_bytes, uint64_t max_grid_cells,
                             cudaStream_t s, Index &ix);
sj_status read_counts(Error &err, Index &ix, cudaStream_t s);
const uint32_t *n_items_dev(const Index &ix);

// Arguments of one search-and-refine launch.
struct JoinArgs {
    // index
    const float *rec32;
    const double *rec64;
    const double *pts;              // original points, FP64 recheck
    const uint32_t *G;
    const uint64_t *B;
    const int32_t *cc;
    const uint32_t *M;
    const uint32_t *lut;
    const uint2 *items;
    // query side: the same index for a self-join; another index on the
    // same grid for a two-set join
    const float *qrec32;
    const double *qrec64;
    const double *qpts;
    const uint32_t *qG;
    const int32_t *qcc;
    const uint32_t *ccells;         // candidate |G| (device)
    uint32_t item_begin, item_end;
    uint32_t item_stride;           // sampled launches: every item_stride-th item
    uint32_t n_cells;
    uint32_t mwords;
    int dense;
    int tuple;                      // cells searched by coordinate tuple (cc), not by B
    int rs;                         // record stride in elements of the mode's type
    int n_templates;
    const uint32_t *tmpl;           // row templates of (d, UNICOMP), device memory
    int32_t ng[kMaxDim];
    uint64_t stride[kMaxDim];
    float lo32, hi32;
    float w32;                      // cell side in the FP32 frame
    float w4, inv_w4;               // cell frame: frame step 4 w32 and its inverse
    int frame;                      // sj_frame of the FP32 records
    double E2;
    int qrs;                        // staged query record stride (elements)
    // output
    uint2 *out;
    uint64_t cap;
    unsigned long long *counter;    // [0] pairs, [1] evaluations, [2] rechecks
    uint32_t *work;                 // work-item cursor
    uint32_t *error;                // device error word
    int count_only;
    int grab;                       // items taken per cursor bump
    // per-warp shared-memory layout (bytes)
    int sm_ranges, sm_queries, sm_chunk, sm_emit, sm_warp;
    int cb;                         // candidates per chunk
    int eb;                         // emission staging entries
    int nbuf;                       // chunk ring depth (2..8)
    int slots;                      // item slots per warp (1 or 2)
    uint64_t timeout_ns;            // limit of each bounded mbarrier wait
    int stall;                      // test hook: warp 0 of block 0 skips its first copy
    // multi-join launches: the dimension and precision of this job and its
    // device counters (|G|, work items) in place of the kernel argument
    int d;
    int f32;
    const uint32_t *dcounts;
    // high-dimensional path: records of all dfull coordinates
    const float *recd32;
    const double *recd64;
    const double *ptsd;
    int dfull;
    int rsd;                        // their stride in elements of the mode's type
    // expanded-form FP32 sum (margin.cu, fp32_margin_hd): nibble j of hgrid4
    // is the grid dimension that dimension j is (15: none); hmid[j] (device
    // memory) the origin of the others
    int hd_exp;
    uint64_t hgrid4;
    const float *hmid;
};

struct JoinLaunch {
    int prec_fp32 = 1;
    int unicomp = 1;
    int blocks = 0;                 // 0: derive from occupancy
    int grab = 0;
    uint32_t item_stride = 1;
    int wpb = 0;                    // warps per block; 0: occupancy picks
    int nbuf = 0;                   // chunk ring depth; 0: by dimension and precision
    int eb = 0;                     // staged pairs per warp (128..1024); 0: by dimension
    int slots = 0;                  // item slots per warp (1 or 2); 0: by dimension
    uint64_t timeout_ns = 0;        // bounded waits; 0: 2 s
    int stall = 0;                  // test hook (sj_config.test_stall)
};

// Job table of a multi-join launch, passed in the kernel parameters.
constexpr int kMultiJobs = 64;
struct MultiJobs {
    uint32_t n;
    uint32_t pad;
    JoinArgs job[kMultiJobs];
};
static_assert(sizeof(MultiJobs) <= 32000, "multi-join table exceeds the kernel parameter limit");

// A search-and-refine kernel: (arguments, device counters |G| and items).
typedef void (*JoinKernelFn)(const JoinArgs, const uint32_t *);
// The kernel for points of d = 9..16 dimensions (hd_join.cu), null otherwise.
JoinKernelFn hd_kernel_fn(int d, bool f32, bool uni, bool exp);

sj_status fill_join_args(Error &err, const Index &ix, const JoinLaunch &cfg, uint32_t item_begin,
                         uint32_t item_end, uint2 *out, uint64_t cap,
                         unsigned long long *d_counter, uint32_t *d_work, uint32_t *d_error,
                         int count_only, JoinArgs &a, const Index *qix = nullptr);
sj_status block_shape(Error &err, const void *fn, int sm_warp, int force_wpb, int dev, int *wpb,
                      int *per_sm);
// Index-free comparator (brute.cu): every ordered pair with the exact FP64
// predicate; *d_counter accumulates the member count.
sj_status brute_join(Error &err, const double *d_pts, uint64_t n, int d, double eps, uint2 *out,
                     uint64_t cap, unsigned long long *d_counter, cudaStream_t s);
// Work-item range [lo, hi) of shard `rank` of `world` (shard.cu): equal
// shares of the estimated search cost, each bound moved forward to a cell
// start.  Synchronises s.
sj_status shard_items(Error &err, const Index &ix, bool uni, int rank, int world, cudaStream_t s,
                      uint32_t *lo, uint32_t *hi);
// Launch tuner (tune.cu): on a miss times sampled count-only launches of ix
// and stores the fastest (grab, ring depth, warps per block) for the key
// (d, precision, UNICOMP, points-per-cell bucket); *tuned = 0 defaults kept,
// 1 taken from the cache, 2 tuned now.  ix.n_cells must be known on the
// host; a miss reads the work-item count first (read_counts).
// True when the configuration forces a launch parameter (the tuners then
// keep out).
bool launch_forced(const sj_config &c);
int tune_bucket(const Index &ix);
int tune_bucket_ppc(double points_per_cell);
// Smallest join (work items) the tuner times; smaller joins keep the defaults.
constexpr uint32_t kTuneMinItems = 4096;
sj_status tune_launch(Error &err, Index &ix, JoinLaunch &l, cudaStream_t s, int *tuned);
void tune_clear();
// The multi-join kernel (join.cu): void(const MultiJobs).
const void *multi_join_fn();
// Geometry of Section IV-B from per-dimension bounds (index.cu).
sj_status geometry_from_bounds(Error &err, const unsigned long long *mm, int d, uint64_t n,
                               double eps, int frame_mode, Geometry &g);
int n_templates(int d, bool uni);

// qix: the query-side index of a two-set join (same grid as ix), else null.
sj_status launch_join(Error &err, const Index &ix, const JoinLaunch &cfg, uint32_t item_begin,
                      uint32_t item_end, uint2 *out, uint64_t cap,
                      unsigned long long *d_counter, uint32_t *d_work, uint32_t *d_error,
                      int count_only, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                      const Index *qix = nullptr);

// Device-wide exclusive scan of u32 (in may equal out).  *d_total receives the
// sum.  Returns SJ_OK or an error.
sj_status exclusive_scan_u32(Error &err, const uint32_t *in, uint32_t *out, uint64_t n,
                             uint32_t *d_total, cudaStream_t s);
// The same with caller-provided tile sums (n up to 4096^2).
uint64_t scan_sums_needed(uint64_t n);
sj_status exclusive_scan_u32_scratch(Error &err, const uint32_t *in, uint32_t *out, uint64_t n,
                                     uint32_t *d_total, uint32_t *sums, uint64_t sums_cap,
                                     cudaStream_t s);

// Stable LSD radix sort of (key, value) by the low `bits` bits of key.
sj_status radix_sort_pairs(Error &err, uint64_t *keys, uint32_t *vals, uint64_t n, int bits,
                           cudaStream_t s);

// Host helpers
double now_ms();
// Counts kernel launches of the library (read per call into sj_stats).
void note_launch();
uint64_t launches_so_far();
int sm_count(int device);

// Pinned host memory shared by all contexts (api.cu).
void *pinned_get(size_t bytes, size_t *got);
void pinned_put(void *p, size_t bytes);

}  // namespace sj

// ---------------------------------------------------------------- opaque types

struct sj_result {
    uint32_t *pairs = nullptr;
    uint64_t count = 0;
    size_t bytes = 0;     // capacity of the pinned buffer
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct sj_index {
    sj::Index ix;
    int device = 0;
};

struct sj_ctx {
    sj_config cfg;
    int device = 0;
    cudaStream_t s_main = nullptr, s_copy = nullptr;
    sj::DevBuf misc;                         // join counters, work cursor, error word
    unsigned long long *h_misc = nullptr;    // pinned read-back (64 words)
    cudaEvent_t ev_counts = nullptr;         // build counters copied to h_misc (BuildOpts)
    std::string last_err;
    sj_stats stats;
    double t0 = 0;
    // profiling
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
    size_t prof_used = 0;
    double prof_ms = 0;
    uint64_t prof_launches = 0;
    // launch parameters of the current join (defaults or the tuner's)
    sj::JoinLaunch launch;
    int launch_tuned = 0;
    // serving scheduler (serve.cu) and the multi-join engine of
    // sj_selfjoin_multi (engine.cu)
    void *serve = nullptr;
    void *engine = nullptr;
};

namespace sj {
// Sorts a host result ascending by (i << 32) | j (api.cu).
void sort_result(sj_result *r);
}  // namespace sj
