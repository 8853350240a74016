// engine.cu -- many self-joins in one pass.
//
// A wave is a set of up to kMultiJobs independent joins (each with its own
// n, d and eps).  It runs as
//   1. the points of every job to the device and one bounds launch over all
//      jobs, then ONE host read-back of all bounds (the geometry of Section
//      IV-B and the FP32 margin are derived on the host, as in index.cu);
//   2. one replay of the engine's CUDA graph: the index build of Section
//      IV-B/C for all jobs at once (every build kernel covers every job: the
//      blocks of its fixed grid are shared out to the jobs in proportion to
//      their size by a table in device memory), then one persistent
//      multi-join launch (join.cu) in which every warp works through the
//      jobs' work items, job after job;
//   3. one read-back of all pair counts, and the pairs of every job to
//      pinned host memory.
// The graph is captured once per engine: all build kernels read their job
// table from device memory, so only the multi-join node's launch shape and
// job table (kernel parameters) are updated per wave.
//
// Launch parameters: the context's forced ones, else those of the wave
// tuner, else the defaults.  The wave tuner times the multi-join launch of
// a wave itself, not single joins: the choices of the single-join tuner
// (tune.cu) lost in one launch of many small joins (measured on the
// 10,000-request stream, passes interleaved: 0.90x of the fixed defaults
// with the tuned grab alone; 9.3 against 12.9 G pairs/s with every tuned
// parameter, since one job's larger shared memory per warp lowers the
// occupancy of the whole wave).  The first wave of a key (precision,
// log2 of the wave's points per SM) is re-joined with each candidate
// setting, applied to every job of the wave (the work items a warp takes
// per cursor bump, the candidate-chunk ring depth, the pair staging size,
// the item slots), one parameter after another; a change is kept when
// its launch is at least 3% faster.  Every timed launch writes the whole
// result again, so the wave's result is that of the last one.  Timing
// needs the GPU alone: the waves of all engines of the process hold a
// shared gate for their graph replay and a tuning pass holds it
// exclusively (a waiting pass holds back new waves).
//
// The engine takes jobs whose grid fits the dense lookup table (at most
// max(2^25, 16 n) cells, and at most kEngMaxLut) with n <= kEngMaxN; any
// other job runs through the stand-alone path of a private context.  The
// result buffer of a job is sized from an estimate of its pair count; a job
// whose pairs overflow it (the kernel still counts them all) is joined again
// alone into a buffer of the exact size, using the index already built.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "engine.cuh"
#include "grid_dev.cuh"

namespace sj {

namespace {

constexpr int kEngThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kEngThreads * kScanPer;          // 4096 values per scan tile
constexpr uint32_t kMaxScanTiles = 16384;
constexpr uint64_t kEngMaxLut = (uint64_t)kScanTile * kMaxScanTiles;   // 2^26 cells
constexpr uint64_t kEngMaxN = (uint64_t)kScanTile * kMaxScanTiles;     // 2^26 points
constexpr int kMmWords = 2 * kMaxDim + 8;   // bounds (order keys) + 16 u32 counters
constexpr int kMiscWords = 8;               // pairs, evaluations, rechecks, -, cursor, error
constexpr int kScanLut = 0, kScanHead = 1, kScanItems = 2;

// Per-job view of the device arrays, read by the build kernels.
struct EngSlot {
    CellParams cp;
    const double *pts;
    uint64_t n;
    uint64_t lut_len;            // grid cells + 1
    uint32_t mwords;
    int rs32, rs64, need64;
    unsigned long long *mm;      // bounds; the counters follow
    uint32_t *counts;            // [0] non-finite flag, [1] |G|, [2] work items, [3] lut total
    unsigned long long *misc;    // join counters, cursor, error word
    uint32_t *lut;
    uint64_t *key;
    uint32_t *rank;
    uint32_t *A;
    uint64_t *skey;
    uint32_t *head;
    uint64_t *B;
    uint32_t *G;
    int32_t *cc;
    uint32_t *M;
    float *rec32;
    double *rec64;
    uint2 *items;
    uint32_t *icnt;
    uint32_t *sums;
};

struct EngTable {
    uint32_t n_slots;
    uint32_t pad;
    uint32_t share[kMultiJobs + 1];   // blocks [share[s], share[s+1]) serve job s
    EngSlot slot[kMultiJobs];
};

// The job this block serves, its block index x within the job and the
// number X of blocks serving the job; false for a block without a job.
__device__ __forceinline__ bool my_slot(const EngTable *__restrict__ t, uint32_t &s, uint32_t &x,
                                        uint32_t &X) {
    const uint32_t ns = t->n_slots;
    const uint32_t b = blockIdx.x;
    if (ns == 0 || b >= t->share[ns]) return false;
    uint32_t lo = 0, hi = ns;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (t->share[mid] <= b) lo = mid; else hi = mid;
    }
    s = lo;
    x = b - t->share[lo];
    X = t->share[lo + 1] - t->share[lo];
    return X > 0;
}

// Exclusive scan over the threads of a block (blockDim a multiple of 32, at
// most 1024); *total receives the block's sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t wsum[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = lane < nw ? wsum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    const uint32_t r = wsum[wid] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return r;
}

__global__ void eng_bounds_init(const EngTable *__restrict__ t) {
    const uint32_t s = threadIdx.x;
    if (s >= t->n_slots) return;
    unsigned long long *mm = t->slot[s].mm;
    for (int j = 0; j < kMaxDim; ++j) {
        mm[2 * j] = ~0ULL;
        mm[2 * j + 1] = 0ULL;
    }
    for (int k = 0; k < 16; ++k) t->slot[s].counts[k] = 0;
}

__global__ void __launch_bounds__(kEngThreads) eng_bounds(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    bounds_accumulate(e.pts, e.n, e.cp.d, (uint64_t)x * blockDim.x + threadIdx.x,
                      (uint64_t)X * blockDim.x, e.mm, e.counts);
}

// Clears what the build accumulates into: the dense table, M_j, the join
// counters and the build counters (the non-finite flag is kept).
__global__ void __launch_bounds__(kEngThreads) eng_clear(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const uint64_t i0 = (uint64_t)x * blockDim.x + threadIdx.x, step = (uint64_t)X * blockDim.x;
    for (uint64_t i = i0; i < e.lut_len; i += step) e.lut[i] = 0u;
    const uint64_t mw = (uint64_t)e.cp.d * e.mwords;
    for (uint64_t i = i0; i < mw; i += step) e.M[i] = 0u;
    if (i0 < kMiscWords) e.misc[i0] = 0ull;
    if (i0 >= 1 && i0 < 16) e.counts[i0] = 0u;
}

// Cell id of every point and its rank inside the cell (counting sort).
__global__ void __launch_bounds__(kEngThreads) eng_cell(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const CellParams cp = e.cp;
    for (uint64_t i = (uint64_t)x * blockDim.x + threadIdx.x; i < e.n; i += (uint64_t)X * blockDim.x) {
        const uint64_t id = linear_cell(e.pts + i * cp.d, cp);
        e.key[i] = id;
        e.rank[i] = atomicAdd(&e.lut[id], 1u);
    }
}

template <int MODE>
__device__ __forceinline__ uint64_t scan_len(const EngSlot &e) {
    return MODE == kScanLut ? e.lut_len : e.n;
}

// Value k of the scanned sequence: cell counts, cell-head flags of the
// sorted keys, or work items per non-empty cell.
template <int MODE>
__device__ __forceinline__ uint32_t scan_val(const EngSlot &e, uint64_t k, uint32_t n_cells) {
    if (MODE == kScanLut) return e.lut[k];
    if (MODE == kScanHead) return (k == 0 || e.skey[k] != e.skey[k - 1]) ? 1u : 0u;
    return k < n_cells ? (e.G[k + 1] - e.G[k] + kQueryBlock - 1) / kQueryBlock : 0u;
}

template <int MODE>
__device__ __forceinline__ uint32_t *scan_out(const EngSlot &e) {
    return MODE == kScanLut ? e.lut : (MODE == kScanHead ? e.head : e.icnt);
}

// counts[] index of the scan's total: lut total, |G|, work items
template <int MODE>
__device__ __forceinline__ int scan_total_at() {
    return MODE == kScanLut ? 3 : (MODE == kScanHead ? 1 : 2);
}

// Scan phase 1: the sum of every tile of 4096 values.
template <int MODE>
__global__ void __launch_bounds__(kEngThreads) eng_scan_reduce(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const uint64_t L = scan_len<MODE>(e);
    const uint32_t T = (uint32_t)((L + kScanTile - 1) / kScanTile);
    const uint32_t nc = MODE == kScanItems ? e.counts[1] : 0u;
    for (uint32_t tile = x; tile < T; tile += X) {
        const uint64_t base = (uint64_t)tile * kScanTile;
        uint32_t v = 0;
#pragma unroll 4
        for (int i = 0; i < kScanPer; ++i) {
            const uint64_t k = base + (uint64_t)i * kEngThreads + threadIdx.x;
            if (k < L) v += scan_val<MODE>(e, k, nc);
        }
        uint32_t tot;
        (void)block_excl_scan(v, &tot);
        if (threadIdx.x == 0) e.sums[tile] = tot;
    }
}

// Scan phase 2: one block per job turns the tile sums into tile offsets
// and stores the total.
template <int MODE>
__global__ void __launch_bounds__(1024) eng_scan_sums(const EngTable *__restrict__ t) {
    const uint32_t s = blockIdx.x;
    if (s >= t->n_slots) return;
    const EngSlot &e = t->slot[s];
    const uint64_t L = scan_len<MODE>(e);
    const uint32_t T = (uint32_t)((L + kScanTile - 1) / kScanTile);
    uint32_t run = 0;
    for (uint32_t base = 0; base < T; base += blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        const uint32_t v = k < T ? e.sums[k] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(v, &tot);
        if (k < T) e.sums[k] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) e.counts[scan_total_at<MODE>()] = run;
}

// Scan phase 3: exclusive prefix of every value (in place for the table).
template <int MODE>
__global__ void __launch_bounds__(kEngThreads) eng_scan_down(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const uint64_t L = scan_len<MODE>(e);
    const uint32_t T = (uint32_t)((L + kScanTile - 1) / kScanTile);
    const uint32_t nc = MODE == kScanItems ? e.counts[1] : 0u;
    uint32_t *out = scan_out<MODE>(e);
    for (uint32_t tile = x; tile < T; tile += X) {
        uint32_t run = e.sums[tile];
        const uint64_t base = (uint64_t)tile * kScanTile;
        for (int i = 0; i < kScanPer; ++i) {
            const uint64_t k = base + (uint64_t)i * kEngThreads + threadIdx.x;
            const uint32_t v = k < L ? scan_val<MODE>(e, k, nc) : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan(v, &tot);
            if (k < L) out[k] = run + ex;
            run += tot;
        }
    }
}

// Counting-sort scatter: A[lut[id] + rank] = i, with the sorted key.
__global__ void __launch_bounds__(kEngThreads) eng_scatter(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    for (uint64_t i = (uint64_t)x * blockDim.x + threadIdx.x; i < e.n; i += (uint64_t)X * blockDim.x) {
        const uint64_t id = e.key[i];
        const uint32_t pos = e.lut[id] + e.rank[i];
        e.A[pos] = (uint32_t)i;
        e.skey[pos] = id;
    }
}

// Run-length compaction: B and G from the scanned head flags.
__global__ void __launch_bounds__(kEngThreads) eng_rle(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    for (uint64_t k = (uint64_t)x * blockDim.x + threadIdx.x; k < e.n; k += (uint64_t)X * blockDim.x) {
        if (k == 0 || e.skey[k] != e.skey[k - 1]) {
            const uint32_t h = e.head[k];
            e.B[h] = e.skey[k];
            e.G[h] = (uint32_t)k;
        }
        if (k == 0) e.G[e.counts[1]] = (uint32_t)e.n;
    }
}

__global__ void __launch_bounds__(kEngThreads) eng_cells(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    __shared__ uint32_t sm[kCellsSmemWords];
    cells_block<true>(e.pts, e.A, e.G, e.B, e.counts[1], (uint64_t)x * blockDim.x + threadIdx.x,
                      (uint64_t)X * blockDim.x, e.cp, e.mwords, e.cc, e.M, sm);
}

__global__ void __launch_bounds__(kEngThreads) eng_rec(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const CellParams cp = e.cp;
    for (uint64_t k = (uint64_t)x * blockDim.x + threadIdx.x; k < e.n; k += (uint64_t)X * blockDim.x) {
        write_rec32(e.pts, e.A, k, cp, e.rs32, e.rec32);
        if (e.need64) write_rec64(e.pts, e.A, k, cp.d, e.rs64, e.rec64);
    }
}

__global__ void __launch_bounds__(kEngThreads) eng_item_fill(const EngTable *__restrict__ t) {
    uint32_t s, x, X;
    if (!my_slot(t, s, x, X)) return;
    const EngSlot &e = t->slot[s];
    const uint32_t nc = e.counts[1];
    for (uint64_t h = (uint64_t)x * blockDim.x + threadIdx.x; h < nc; h += (uint64_t)X * blockDim.x) {
        const uint32_t nb = (e.G[h + 1] - e.G[h] + kQueryBlock - 1) / kQueryBlock;
        const uint32_t o = e.icnt[h];
        for (uint32_t b = 0; b < nb; ++b) e.items[o + b] = make_uint2((uint32_t)h, b);
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Splits `blocks` blocks over k jobs: at least one each, the rest in
// proportion to the weights; writes the prefix into share[0..k].
void share_blocks(uint32_t *share, const std::vector<double> &w, int blocks) {
    const int k = (int)w.size();
    double W = 0;
    for (double v : w) W += v;
    const int spare = std::max(0, blocks - k);
    share[0] = 0;
    for (int s = 0; s < k; ++s) {
        const uint32_t extra = W > 0 ? (uint32_t)std::floor(spare * (w[s] / W)) : 0u;
        share[s + 1] = share[s] + 1 + extra;
    }
}

double ball_volume(int d) { return std::pow(M_PI, 0.5 * d) / std::tgamma(0.5 * d + 1.0); }

// Ordered pairs (self-pairs included) expected for n points spread
// uniformly over a box of the given side lengths.
double uniform_pairs(uint64_t n, int d, double eps, const double *side) {
    double vol = 1.0;
    for (int j = 0; j < d; ++j) vol *= std::max(side[j], eps);
    double nb = (double)(n - 1) * ball_volume(d) * std::pow(eps, d) / vol;
    nb = std::min(nb, (double)(n - 1));
    return (double)n * (1.0 + nb);
}

}  // namespace

class Engine {
public:
    int device = 0;
    sj_config cfg;
    cudaStream_t st = nullptr;
    EngTable *d_table = nullptr, *h_table = nullptr;
    unsigned long long *d_mm = nullptr, *h_mm = nullptr;
    unsigned long long *d_misc = nullptr, *h_misc = nullptr;
    MultiJobs *h_mj = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t join_node = nullptr;
    int build_blocks = 0;
    int sms = 0;
    sj_ctx *fallback = nullptr;
    cudaEvent_t ev[kMultiJobs] = {};   // per-job completion of the result copies
    EngStats stats;
};

namespace {

sj_status capture_graph(Error &err, Engine *e) {
    const EngTable *t = e->d_table;
    const int B = e->build_blocks;
    cudaStream_t s = e->st;
    SJ_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    eng_clear<<<B, kEngThreads, 0, s>>>(t);
    eng_cell<<<B, kEngThreads, 0, s>>>(t);
    eng_scan_reduce<kScanLut><<<B, kEngThreads, 0, s>>>(t);
    eng_scan_sums<kScanLut><<<kMultiJobs, 1024, 0, s>>>(t);
    eng_scan_down<kScanLut><<<B, kEngThreads, 0, s>>>(t);
    eng_scatter<<<B, kEngThreads, 0, s>>>(t);
    eng_scan_reduce<kScanHead><<<B, kEngThreads, 0, s>>>(t);
    eng_scan_sums<kScanHead><<<kMultiJobs, 1024, 0, s>>>(t);
    eng_scan_down<kScanHead><<<B, kEngThreads, 0, s>>>(t);
    eng_rle<<<B, kEngThreads, 0, s>>>(t);
    eng_cells<<<B, kEngThreads, 0, s>>>(t);
    eng_rec<<<B, kEngThreads, 0, s>>>(t);
    eng_scan_reduce<kScanItems><<<B, kEngThreads, 0, s>>>(t);
    eng_scan_sums<kScanItems><<<kMultiJobs, 1024, 0, s>>>(t);
    eng_scan_down<kScanItems><<<B, kEngThreads, 0, s>>>(t);
    eng_item_fill<<<B, kEngThreads, 0, s>>>(t);
    // the join node: an empty job table now, set per wave
    std::memset(e->h_mj, 0, sizeof(MultiJobs));
    void *args[] = {e->h_mj};
    cudaError_t le = cudaLaunchKernel(multi_join_fn(), dim3(1), dim3(32), args, 0, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); SJ_CUDA_TRY(le); }
    SJ_CUDA_TRY(ce);
    e->graph = g;
    SJ_CUDA_TRY(cudaGraphInstantiate(&e->exec, g, 0));
    size_t nn = 0;
    SJ_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    SJ_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
    int kernels = 0;
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType ty;
        SJ_CUDA_TRY(cudaGraphNodeGetType(n, &ty));
        if (ty != cudaGraphNodeTypeKernel) continue;
        ++kernels;
        cudaKernelNodeParams kp;
        SJ_CUDA_TRY(cudaGraphKernelNodeGetParams(n, &kp));
        if (kp.func == multi_join_fn()) e->join_node = n;
    }
    if (!e->join_node) return fail(err, SJ_ECUDA, "multi-join node not found in the captured graph");
    e->stats.kernel_nodes = (uint64_t)kernels;
    return SJ_OK;
}

// Device pointers of a job's arrays, carved from one allocation.
struct JobMem {
    DevBuf pts, region, out2;
    uint64_t cap = 0;            // pairs the result buffer holds
    uint2 *out = nullptr;
    Geometry g;
    Index view;                  // non-owning view for fill_join_args / launch_join
    bool f32 = true;
    uint64_t lut_len = 0;
    double est = 0;
    int row = 0;                 // bounds / counter row
    const uint2 *src = nullptr;  // pairs to copy out
    uint64_t count = 0;
};

}  // namespace

sj_status engine_create(Error &err, int device, const sj_config &cfg, Engine **out) {
    *out = nullptr;
    Engine *e = new Engine();
    e->device = device;
    e->cfg = cfg;
    auto bad = [&](sj_status st) {
        engine_destroy(e);
        return st;
    };
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) { set_cuda_error(err, ce, "cudaSetDevice", __FILE__, __LINE__); return bad(err.st); }
    e->sms = sm_count(device);
    e->build_blocks = 8 * e->sms;
    if ((ce = cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_table, sizeof(EngTable))) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_mm, sizeof(unsigned long long) * kMultiJobs * kMmWords)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_misc, sizeof(unsigned long long) * kMultiJobs * kMiscWords)) != cudaSuccess ||
        (ce = cudaHostAlloc(&e->h_table, sizeof(EngTable), cudaHostAllocPortable)) != cudaSuccess ||
        (ce = cudaHostAlloc(&e->h_mm, sizeof(unsigned long long) * kMultiJobs * kMmWords,
                            cudaHostAllocPortable)) != cudaSuccess ||
        (ce = cudaHostAlloc(&e->h_misc, sizeof(unsigned long long) * kMultiJobs * kMiscWords,
                            cudaHostAllocPortable)) != cudaSuccess) {
        set_cuda_error(err, ce, "engine allocation", __FILE__, __LINE__);
        return bad(SJ_ENOMEM);
    }
    for (int q = 0; q < kMultiJobs; ++q)
        if ((ce = cudaEventCreateWithFlags(&e->ev[q], cudaEventDisableTiming)) != cudaSuccess) {
            set_cuda_error(err, ce, "cudaEventCreate", __FILE__, __LINE__);
            return bad(err.st);
        }
    e->h_mj = static_cast<MultiJobs *>(std::calloc(1, sizeof(MultiJobs)));
    if (!e->h_mj) return bad(fail(err, SJ_ENOMEM, "host allocation failed"));
    std::memset(e->h_table, 0, sizeof(EngTable));
    if ((ce = cudaMemcpy(e->d_table, e->h_table, sizeof(EngTable), cudaMemcpyHostToDevice)) != cudaSuccess) {
        set_cuda_error(err, ce, "cudaMemcpy", __FILE__, __LINE__);
        return bad(err.st);
    }
    const sj_status st = capture_graph(err, e);
    if (st != SJ_OK) return bad(st);
    *out = e;
    return SJ_OK;
}

void engine_destroy(Engine *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->st) cudaStreamSynchronize(e->st);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->d_table) cudaFree(e->d_table);
    if (e->d_mm) cudaFree(e->d_mm);
    if (e->d_misc) cudaFree(e->d_misc);
    if (e->h_table) cudaFreeHost(e->h_table);
    if (e->h_mm) cudaFreeHost(e->h_mm);
    if (e->h_misc) cudaFreeHost(e->h_misc);
    std::free(e->h_mj);
    for (int q = 0; q < kMultiJobs; ++q)
        if (e->ev[q]) cudaEventDestroy(e->ev[q]);
    if (e->fallback) sj_destroy(e->fallback);
    if (e->st) cudaStreamDestroy(e->st);
    cudaGetLastError();
    delete e;
}

EngStats engine_stats(const Engine *e) { return e ? e->stats : EngStats(); }

uint64_t engine_estimate(const double *pts, uint64_t n, int d, double eps, uint64_t *pairs) {
    double lo[kMaxDim], hi[kMaxDim], side[kMaxDim];
    for (int j = 0; j < d; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
    const uint64_t m = std::min<uint64_t>(n, 512);
    for (uint64_t t = 0; t < m; ++t) {
        const uint64_t i = (m == n) ? t : (t * (n - 1)) / (m - 1 ? m - 1 : 1);
        for (int j = 0; j < d; ++j) {
            const double x = pts[i * d + j];
            lo[j] = std::min(lo[j], x);
            hi[j] = std::max(hi[j], x);
        }
    }
    const double w = eps * (1.0 + std::ldexp(1.0, -16));
    double cells = 1.0;
    for (int j = 0; j < d; ++j) {
        side[j] = std::isfinite(hi[j] - lo[j]) ? hi[j] - lo[j] : 0.0;
        cells *= std::floor((side[j] + 2 * eps) / w) + 1.0;
    }
    const double p = uniform_pairs(n, d, eps, side);
    if (pairs) *pairs = (uint64_t)p;
    const int rs32 = (d + 1 + 3) / 4 * 4;
    const double per_point = 8.0 * d + 56 + 4.0 * d + 4.0 * rs32;
    const double lut = 4.0 * std::min(cells * 1.5, std::max((double)(1 << 25), 16.0 * n));
    return (uint64_t)(per_point * n + lut + 8.0 * (1.25 * p + 4096) + (1 << 20));
}

namespace {

// Launch parameters of the wave tuner, applied to every job of a wave.
struct WaveTune {
    int grab = 1, nbuf = 0, eb = 0, slots = 0;
};

// Waves below this many points are not tuned: their launch is too short to
// time apart from noise.
constexpr uint64_t kWaveTuneMinPoints = 1ull << 17;

std::mutex g_wave_mu;
std::map<std::pair<int, int>, WaveTune> g_wave_tuned;   // (precision, bucket) -> choice
std::set<std::pair<int, int>> g_wave_pending;           // keys a tuning pass is working on

// The GPU gate of the waves of every engine of the process: waves hold it
// shared for their graph replay, a tuning pass exclusively.  A waiting
// tuning pass holds back new shared holders, so that it is not starved by
// overlapping waves.
class GpuGate {
public:
    void lock_shared() {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return !writer_ && waiting_ == 0; });
        ++readers_;
    }
    void unlock_shared() {
        std::lock_guard<std::mutex> lk(mu_);
        if (--readers_ == 0) cv_.notify_all();
    }
    void lock() {
        std::unique_lock<std::mutex> lk(mu_);
        ++waiting_;
        cv_.wait(lk, [&] { return !writer_ && readers_ == 0; });
        --waiting_;
        writer_ = true;
    }
    void unlock() {
        std::lock_guard<std::mutex> lk(mu_);
        writer_ = false;
        cv_.notify_all();
    }

private:
    std::mutex mu_;
    std::condition_variable cv_;
    int readers_ = 0, waiting_ = 0;
    bool writer_ = false;
};
GpuGate g_gate;

// Key of a wave: (precision, round(log2(points of the wave per SM))).
std::pair<int, int> wave_key(const Engine *e, uint64_t points) {
    const double per_sm = (double)points / (double)std::max(1, e->sms);
    return std::make_pair(e->cfg.prec == SJ_PREC_FP32_RECHECK ? 1 : 0,
                          (int)std::lround(std::log2(std::max(1.0, per_sm))));
}

// Launch parameters of a job: the context's forced ones, else the wave
// tuner's choice t (when given), else the defaults.
JoinLaunch job_launch(const Engine *e, const WaveTune *t = nullptr) {
    JoinLaunch l;
    l.prec_fp32 = e->cfg.prec == SJ_PREC_FP32_RECHECK;
    l.unicomp = 1;
    if (launch_forced(e->cfg) || !t) {
        l.grab = e->cfg.grab > 0 ? e->cfg.grab : 1;
        l.nbuf = e->cfg.nbuf > 0 ? e->cfg.nbuf : 0;
        l.eb = e->cfg.staging > 0 ? e->cfg.staging : 0;
        l.slots = e->cfg.slots > 0 ? e->cfg.slots : 0;
    } else {
        l.grab = t->grab;
        l.nbuf = t->nbuf;
        l.eb = t->eb;
        l.slots = t->slots;
    }
    return l;
}

// The tuning pass of a wave whose graph replay has finished (the jobs in
// `order` are built and joined): times the multi-join launch over the whole
// wave with candidate settings, one parameter after another, and returns
// the best in *best (*ok false when a timed launch failed: the defaults
// are then launched once more, so that the wave still ends with a complete
// result).  Each timed launch clears the jobs' counters and writes every
// result again.
sj_status tune_wave(Error &err, Engine *e, const std::vector<int> &order, std::vector<JobMem> &mem,
                    WaveTune *best, bool *ok) {
    cudaStream_t s = e->st;
    MultiJobs *MJ = e->h_mj;
    const int nj = (int)order.size();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    SJ_CUDA_TRY(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(ev[0]);
        return fail(err, SJ_ECUDA, "cudaEventCreate failed");
    }
    auto time_it = [&](const WaveTune &t, double *ms) -> sj_status {
        const JoinLaunch l = job_launch(e, &t);
        int smw = 0;
        for (int q = 0; q < nj; ++q) {
            const int i = order[q];
            unsigned long long *misc = e->d_misc + (size_t)i * kMiscWords;
            SJ_TRY(fill_join_args(err, mem[i].view, l, 0, 0xffffffffu, mem[i].out, mem[i].cap, misc,
                                  reinterpret_cast<uint32_t *>(misc + 4),
                                  reinterpret_cast<uint32_t *>(misc + 5), 0, MJ->job[q]));
            smw = std::max(smw, MJ->job[q].sm_warp);
        }
        for (int q = 0; q < nj; ++q) MJ->job[q].sm_warp = smw;
        MJ->n = (uint32_t)nj;
        int wpb = 0, per_sm = 0;
        SJ_TRY(block_shape(err, multi_join_fn(), smw, 0, e->device, &wpb, &per_sm));
        SJ_CUDA_TRY(cudaMemsetAsync(e->d_misc, 0, sizeof(unsigned long long) * kMultiJobs * kMiscWords, s));
        void *args[] = {MJ};
        SJ_CUDA_TRY(cudaEventRecord(ev[0], s));
        SJ_CUDA_TRY(cudaLaunchKernel(multi_join_fn(), dim3((unsigned)(per_sm * e->sms)),
                                     dim3((unsigned)(wpb * 32)), args, (size_t)smw * wpb, s));
        note_launch();
        SJ_CUDA_TRY(cudaEventRecord(ev[1], s));
        SJ_CUDA_TRY(cudaEventSynchronize(ev[1]));
        float t_ms = 0;
        SJ_CUDA_TRY(cudaEventElapsedTime(&t_ms, ev[0], ev[1]));
        *ms = t_ms;
        return SJ_OK;
    };
    WaveTune cur;   // the defaults
    double t_cur = 0;
    sj_status st = time_it(cur, &t_cur);
    auto try_one = [&](WaveTune c) {
        if (st != SJ_OK) return;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) {
            cur = c;
            t_cur = t;
        }
    };
    const int grabs[] = {2, 4, 8};
    for (int g : grabs) { WaveTune c = cur; c.grab = g; try_one(c); }
    const int nbufs[] = {2, 3, 4};
    for (int nb : nbufs) { WaveTune c = cur; c.nbuf = nb; try_one(c); }
    const int ebs[] = {256, 512, 1024};
    for (int eb : ebs) { WaveTune c = cur; c.eb = eb; try_one(c); }
    const int slotss[] = {1, 2};
    for (int sl : slotss) { WaveTune c = cur; c.slots = sl; try_one(c); }
    *ok = st == SJ_OK;
    if (st != SJ_OK) {
        // the wave must still end with a complete result: the defaults once more
        cudaGetLastError();
        err = Error();
        double t = 0;
        cur = WaveTune();
        st = time_it(cur, &t);
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    *best = cur;
    return st;
}

sj_status engine_run_impl(Error &err, Engine *e, EngJob *const *jobs, int k,
                          void (*on_done)(void *user, int job), void *user,
                          std::vector<JobMem> &mem) {
    SJ_CUDA_TRY(cudaSetDevice(e->device));
    cudaStream_t s = e->st;
    const double t0 = now_ms();
    std::vector<int> standalone;
    for (int i = 0; i < k; ++i) {
        jobs[i]->st = SJ_OK;
        jobs[i]->msg.clear();
        jobs[i]->res = nullptr;
        jobs[i]->evaluations = jobs[i]->rechecks = 0;
        jobs[i]->path = 0;
    }
    auto job_fail = [&](int i, sj_status st, const std::string &msg) {
        jobs[i]->st = st;
        jobs[i]->msg = msg;
    };

    // 1. points and bounds of every job
    std::vector<int> live;
    for (int i = 0; i < k; ++i) {
        EngJob &J = *jobs[i];
        if (!J.pts || J.n == 0 || J.d < 1 || J.d > kMaxDim || !(J.eps > 0.0) || !std::isfinite(J.eps)) {
            job_fail(i, SJ_EINVAL, "invalid argument (pts, n > 0, d in [1,8], eps > 0 finite)");
            continue;
        }
        if (J.n >= (1ull << 32)) { job_fail(i, SJ_ERANGE, "n must be below 2^32"); continue; }
        if (J.n > kEngMaxN) { standalone.push_back(i); continue; }
        Error e2;
        if (dev_alloc(e2, mem[i].pts, J.n * J.d * sizeof(double), s) != SJ_OK) {
            job_fail(i, SJ_ENOMEM, e2.msg);
            continue;
        }
        const cudaError_t ce = cudaMemcpyAsync(mem[i].pts.p, J.pts, J.n * J.d * sizeof(double),
                                               cudaMemcpyDefault, s);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            job_fail(i, SJ_ECUDA, cudaGetErrorString(ce));
            continue;
        }
        live.push_back(i);
    }
    EngTable *T = e->h_table;
    {
        std::vector<double> w;
        for (size_t m = 0; m < live.size(); ++m) {
            const int i = live[m];
            EngSlot &sl = T->slot[m];
            std::memset(&sl, 0, sizeof(sl));
            sl.pts = static_cast<const double *>(mem[i].pts.p);
            sl.n = jobs[i]->n;
            sl.cp.d = jobs[i]->d;
            sl.mm = e->d_mm + (size_t)i * kMmWords;
            sl.counts = reinterpret_cast<uint32_t *>(sl.mm + 2 * kMaxDim);
            mem[i].row = i;
            w.push_back((double)jobs[i]->n);
        }
        T->n_slots = (uint32_t)live.size();
        share_blocks(T->share, w, e->build_blocks);
    }
    if (!live.empty()) {
        const size_t tb = offsetof(EngTable, slot) + live.size() * sizeof(EngSlot);
        SJ_CUDA_TRY(cudaMemcpyAsync(e->d_table, T, tb, cudaMemcpyHostToDevice, s));
        eng_bounds_init<<<1, kMultiJobs, 0, s>>>(e->d_table); note_launch();
        eng_bounds<<<e->build_blocks, kEngThreads, 0, s>>>(e->d_table); note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        SJ_CUDA_TRY(cudaMemcpyAsync(e->h_mm, e->d_mm, sizeof(unsigned long long) * kMultiJobs * kMmWords,
                                    cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const double t1 = now_ms();

    // 2. geometry, memory and job tables
    std::vector<int> run;
    for (int i : live) {
        EngJob &J = *jobs[i];
        JobMem &m = mem[i];
        const unsigned long long *mm = e->h_mm + (size_t)i * kMmWords;
        if (reinterpret_cast<const uint32_t *>(mm + 2 * kMaxDim)[0] & 1u) {
            job_fail(i, SJ_EINVAL, "non-finite coordinate");
            continue;
        }
        Error e2;
        const sj_status gs = geometry_from_bounds(e2, mm, J.d, J.n, J.eps, e->cfg.frame, m.g);
        if (gs != SJ_OK) { job_fail(i, gs, e2.msg); continue; }
        uint64_t dense_limit = std::max<uint64_t>(16 * J.n, 1ull << 25);
        if (m.g.grid_cells > dense_limit || m.g.grid_cells + 1 > kEngMaxLut) {
            standalone.push_back(i);
            continue;
        }
        run.push_back(i);
    }
    std::vector<double> weight;
    int sm_warp_max = 0;
    MultiJobs *MJ = e->h_mj;
    MJ->n = 0;
    // larger joins first, so that the small ones fill the tail of the launch
    for (int i : run) {
        const Geometry &g = mem[i].g;
        double side[kMaxDim];
        for (int j = 0; j < g.d; ++j) side[j] = g.gmax[j] - g.gmin[j] - 2 * g.eps;
        mem[i].est = uniform_pairs(g.n, g.d, g.eps, side);
    }
    std::stable_sort(run.begin(), run.end(), [&](int a, int b) { return mem[a].est > mem[b].est; });
    // the wave tuner: the choice for this wave's key, else (first wave of
    // the key) a tuning pass after the graph replay
    uint64_t wave_points = 0;
    for (int i : run) wave_points += jobs[i]->n;
    const std::pair<int, int> wkey = wave_key(e, wave_points);
    WaveTune wt;
    bool have_wt = false, tune_now = false;
    if (e->cfg.autotune && !launch_forced(e->cfg) && wave_points >= kWaveTuneMinPoints) {
        std::lock_guard<std::mutex> lk(g_wave_mu);
        auto it = g_wave_tuned.find(wkey);
        if (it != g_wave_tuned.end()) {
            wt = it->second;
            have_wt = true;
        } else if (!g_wave_pending.count(wkey)) {
            g_wave_pending.insert(wkey);
            tune_now = true;
        }
    }
    // a pending key is released on every path out of this wave
    struct PendingRelease {
        std::pair<int, int> k;
        bool on;
        ~PendingRelease() {
            if (!on) return;
            std::lock_guard<std::mutex> lk(g_wave_mu);
            g_wave_pending.erase(k);
        }
    } pending_release{wkey, tune_now};
    std::vector<int> order;
    for (int i : run) {
        EngJob &J = *jobs[i];
        JobMem &m = mem[i];
        const Geometry &g = m.g;
        const uint64_t n = J.n;
        const int d = J.d;
        m.f32 = e->cfg.prec == SJ_PREC_FP32_RECHECK && g.fp32_ok;
        m.lut_len = g.grid_cells + 1;
        uint64_t maxng = 1;
        for (int j = 0; j < d; ++j) maxng = std::max<uint64_t>(maxng, (uint64_t)g.ng[j]);
        const uint32_t mwords = (uint32_t)((maxng + 31) / 32);
        const int rs32 = (d + 1 + 3) / 4 * 4, rs64 = (d + 1 + 1) / 2 * 2;
        const uint64_t tiles = (std::max<uint64_t>(m.lut_len, n) + kScanTile - 1) / kScanTile;
        m.cap = (uint64_t)(m.est * 1.25) + 4096;
        // layout: offsets of every array in one allocation
        size_t off = 0;
        auto at = [&](size_t bytes) {
            off = align256(off);
            const size_t o = off;
            off += bytes;
            return o;
        };
        const size_t o_lut = at(m.lut_len * 4), o_key = at(n * 8), o_rank = at(n * 4),
                     o_A = at(n * 4), o_skey = at(n * 8), o_head = at(n * 4), o_B = at(n * 8),
                     o_G = at((n + 1) * 4), o_cc = at(n * d * 4), o_M = at((uint64_t)d * mwords * 4),
                     o_r32 = at(n * rs32 * 4), o_r64 = at(m.f32 ? 0 : n * rs64 * 8),
                     o_items = at(n * 8), o_icnt = at(n * 4), o_sums = at(tiles * 4),
                     o_out = at(m.cap * 8);
        Error e2;
        if (dev_alloc(e2, m.region, align256(off), s) != SJ_OK) {
            job_fail(i, SJ_ENOMEM, e2.msg);
            continue;
        }
        unsigned char *R = static_cast<unsigned char *>(m.region.p);
        const int slot = (int)order.size();
        EngSlot &sl = T->slot[slot];
        std::memset(&sl, 0, sizeof(sl));
        sl.cp = cell_params(g);
        sl.pts = static_cast<const double *>(m.pts.p);
        sl.n = n;
        sl.lut_len = m.lut_len;
        sl.mwords = mwords;
        sl.rs32 = rs32;
        sl.rs64 = rs64;
        sl.need64 = m.f32 ? 0 : 1;
        sl.mm = e->d_mm + (size_t)i * kMmWords;
        sl.counts = reinterpret_cast<uint32_t *>(sl.mm + 2 * kMaxDim);
        sl.misc = e->d_misc + (size_t)i * kMiscWords;
        sl.lut = reinterpret_cast<uint32_t *>(R + o_lut);
        sl.key = reinterpret_cast<uint64_t *>(R + o_key);
        sl.rank = reinterpret_cast<uint32_t *>(R + o_rank);
        sl.A = reinterpret_cast<uint32_t *>(R + o_A);
        sl.skey = reinterpret_cast<uint64_t *>(R + o_skey);
        sl.head = reinterpret_cast<uint32_t *>(R + o_head);
        sl.B = reinterpret_cast<uint64_t *>(R + o_B);
        sl.G = reinterpret_cast<uint32_t *>(R + o_G);
        sl.cc = reinterpret_cast<int32_t *>(R + o_cc);
        sl.M = reinterpret_cast<uint32_t *>(R + o_M);
        sl.rec32 = reinterpret_cast<float *>(R + o_r32);
        sl.rec64 = m.f32 ? nullptr : reinterpret_cast<double *>(R + o_r64);
        sl.items = reinterpret_cast<uint2 *>(R + o_items);
        sl.icnt = reinterpret_cast<uint32_t *>(R + o_icnt);
        sl.sums = reinterpret_cast<uint32_t *>(R + o_sums);
        m.out = reinterpret_cast<uint2 *>(R + o_out);
        // the index view of the join
        Index &v = m.view;
        v = Index();
        v.g = g;
        v.dense = 1;
        v.rs32 = rs32;
        v.rs64 = rs64;
        v.mwords = mwords;
        v.pts.p = m.pts.p;
        v.rec32.p = sl.rec32;
        v.rec64.p = sl.rec64;
        v.A.p = sl.A;
        v.B.p = sl.B;
        v.G.p = sl.G;
        v.cc.p = sl.cc;
        v.M.p = sl.M;
        v.lut.p = sl.lut;
        v.items.p = sl.items;
        v.counts_dev.p = sl.mm;
        const JoinLaunch l = job_launch(e, have_wt ? &wt : nullptr);
        JoinArgs &a = MJ->job[slot];
        if (fill_join_args(e2, v, l, 0, 0xffffffffu, m.out, m.cap, sl.misc,
                           reinterpret_cast<uint32_t *>(sl.misc + 4),
                           reinterpret_cast<uint32_t *>(sl.misc + 5), 0, a) != SJ_OK) {
            job_fail(i, e2.st, e2.msg);
            continue;
        }
        sm_warp_max = std::max(sm_warp_max, a.sm_warp);
        weight.push_back((double)n + (double)m.lut_len / 4.0);
        order.push_back(i);
    }
    const double t2 = now_ms();
    if (!order.empty()) {
        const int nj = (int)order.size();
        MJ->n = (uint32_t)nj;
        for (int q = 0; q < nj; ++q) MJ->job[q].sm_warp = sm_warp_max;
        T->n_slots = (uint32_t)nj;
        share_blocks(T->share, weight, e->build_blocks);
        int wpb = 0, per_sm = 0;
        SJ_TRY(block_shape(err, multi_join_fn(), sm_warp_max, 0, e->device, &wpb, &per_sm));
        const size_t tb = offsetof(EngTable, slot) + nj * sizeof(EngSlot);
        SJ_CUDA_TRY(cudaMemcpyAsync(e->d_table, T, tb, cudaMemcpyHostToDevice, s));
        // the graph replay holds the GPU gate shared (a tuning pass of
        // another engine then waits for it)
        struct SharedHold {
            bool on = false;
            void take() { g_gate.lock_shared(); on = true; }
            void drop() { if (on) g_gate.unlock_shared(); on = false; }
            ~SharedHold() { drop(); }
        } hold;
        hold.take();
        cudaKernelNodeParams kp = {};
        void *args[] = {MJ};
        kp.func = const_cast<void *>(multi_join_fn());
        kp.gridDim = dim3((unsigned)(per_sm * e->sms));
        kp.blockDim = dim3((unsigned)(wpb * 32));
        kp.sharedMemBytes = (unsigned)((size_t)sm_warp_max * wpb);
        kp.kernelParams = args;
        SJ_CUDA_TRY(cudaGraphExecKernelNodeSetParams(e->exec, e->join_node, &kp));
        SJ_CUDA_TRY(cudaGraphLaunch(e->exec, s));
        for (uint64_t q = 0; q < e->stats.kernel_nodes; ++q) note_launch();
        e->stats.graph_launches++;
        if (!tune_now)
            SJ_CUDA_TRY(cudaMemcpyAsync(e->h_misc, e->d_misc,
                                        sizeof(unsigned long long) * kMultiJobs * kMiscWords,
                                        cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        hold.drop();
        if (tune_now) {
            // the first wave of its key: re-joined with each candidate
            // setting while no other wave runs
            const double tt0 = now_ms();
            struct ExclusiveHold {
                ExclusiveHold() { g_gate.lock(); }
                ~ExclusiveHold() { g_gate.unlock(); }
            } excl;
            WaveTune best;
            bool ok = false;
            SJ_TRY(tune_wave(err, e, order, mem, &best, &ok));
            {
                // a pass that failed (ok false) returned the defaults: they
                // are kept for its key, so that the key is not tuned again
                // on every wave
                std::lock_guard<std::mutex> lk(g_wave_mu);
                g_wave_tuned[wkey] = best;
            }
            wt = best;
            e->stats.tuned_waves++;
            e->stats.ms_tune += now_ms() - tt0;
            SJ_CUDA_TRY(cudaMemcpyAsync(e->h_misc, e->d_misc,
                                        sizeof(unsigned long long) * kMultiJobs * kMiscWords,
                                        cudaMemcpyDeviceToHost, s));
            SJ_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    const double t3 = now_ms();
    {
        const JoinLaunch l = job_launch(e, (have_wt || tune_now) ? &wt : nullptr);
        e->stats.last_tuned = tune_now ? 2 : (have_wt ? 1 : 0);
        e->stats.last_grab = l.grab;
        e->stats.last_nbuf = l.nbuf;
        e->stats.last_eb = l.eb;
        e->stats.last_slots = l.slots;
    }

    // 3. counts, reruns after overflow, pairs to the host
    std::vector<int> ready;
    for (int i : order) {
        EngJob &J = *jobs[i];
        JobMem &m = mem[i];
        unsigned long long *h = e->h_misc + (size_t)i * kMiscWords;
        if ((uint32_t)h[5] & kErrTimeout) {
            job_fail(i, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
            continue;
        }
        uint64_t count = h[0];
        J.evaluations = h[1];
        J.rechecks = h[2];
        uint2 *src = m.out;
        if (count > m.cap) {
            // the estimate was short: join this job again alone, exactly sized
            Error e2;
            if (dev_alloc(e2, m.out2, count * 8, s) != SJ_OK) { job_fail(i, SJ_ENOMEM, e2.msg); continue; }
            unsigned long long *dm = e->d_misc + (size_t)i * kMiscWords;
            JoinLaunch l = job_launch(e);
            if (cudaMemsetAsync(dm, 0, kMiscWords * 8, s) != cudaSuccess ||
                launch_join(e2, m.view, l, 0, 0xffffffffu, static_cast<uint2 *>(m.out2.p), count, dm,
                            reinterpret_cast<uint32_t *>(dm + 4), reinterpret_cast<uint32_t *>(dm + 5), 0,
                            s, nullptr, nullptr) != SJ_OK ||
                cudaMemcpyAsync(h, dm, kMiscWords * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                job_fail(i, e2.st != SJ_OK ? e2.st : SJ_ECUDA, e2.msg.empty() ? "rerun failed" : e2.msg);
                continue;
            }
            if ((uint32_t)h[5] & kErrTimeout) {
                job_fail(i, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
                continue;
            }
            if (h[0] != count) { job_fail(i, SJ_ECUDA, "pair count changed between runs"); continue; }
            src = static_cast<uint2 *>(m.out2.p);
            J.path = 2;
            e->stats.overflow_reruns++;
        }
        m.src = src;
        m.count = count;
        ready.push_back(i);
    }
    // pairs to the host, smallest result first, each completing on its own
    // event so that the caller can hand it out before the larger ones land
    std::stable_sort(ready.begin(), ready.end(),
                     [&](int x, int y) { return mem[x].count < mem[y].count; });
    std::vector<int> copied;
    for (int i : ready) {
        sj_result *r = new sj_result();
        size_t got = 0;
        r->pairs = static_cast<uint32_t *>(pinned_get(std::max<size_t>(mem[i].count * 8, 64), &got));
        if (!r->pairs) { delete r; job_fail(i, SJ_ENOMEM, "pinned host allocation failed"); continue; }
        r->bytes = got;
        r->count = mem[i].count;
        cudaError_t ce = cudaMemcpyAsync(r->pairs, mem[i].src, mem[i].count * 8, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e->ev[copied.size()], s);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            pinned_put(r->pairs, r->bytes);
            delete r;
            job_fail(i, SJ_ECUDA, cudaGetErrorString(ce));
            continue;
        }
        jobs[i]->res = r;
        copied.push_back(i);
    }
    std::vector<char> signalled(k, 0);
    for (size_t q = 0; q < copied.size(); ++q) {
        const int i = copied[q];
        const cudaError_t ce = cudaEventSynchronize(e->ev[q]);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            sj_result_free(jobs[i]->res);
            jobs[i]->res = nullptr;
            job_fail(i, SJ_ECUDA, cudaGetErrorString(ce));
        } else if (e->cfg.sorted) {
            sort_result(jobs[i]->res);
        }
        if (on_done) on_done(user, i);
        signalled[i] = 1;
    }
    const double t4 = now_ms();

    // jobs the engine does not take: the stand-alone path
    for (int i : standalone) {
        EngJob &J = *jobs[i];
        if (!e->fallback) {
            sj_config c = e->cfg;
            c.device = e->device;
            const sj_status cs = sj_create(&c, &e->fallback);
            if (cs != SJ_OK) { job_fail(i, cs, "cannot create the stand-alone context"); continue; }
        }
        sj_result *r = nullptr;
        const sj_status js = sj_selfjoin(e->fallback, static_cast<const double *>(J.pts), J.n, J.d,
                                         J.eps, &r);
        if (js != SJ_OK) { job_fail(i, js, sj_last_error(e->fallback)); continue; }
        J.res = r;
        J.path = 1;
        e->stats.standalone++;
    }
    if (on_done)
        for (int i = 0; i < k; ++i)
            if (!signalled[i]) on_done(user, i);
    e->stats.waves++;
    e->stats.jobs += (uint64_t)k;
    e->stats.ms_bounds += t1 - t0;
    e->stats.ms_graph += t3 - t2;
    e->stats.ms_output += t4 - t3;
    return SJ_OK;
}

}  // namespace

sj_status engine_run(Error &err, Engine *e, EngJob *const *jobs, int k,
                     void (*on_done)(void *user, int job), void *user) {
    if (k <= 0) return SJ_OK;
    if (k > kMultiJobs) return fail(err, SJ_EINVAL, "too many jobs for one wave");
    std::vector<JobMem> mem(k);
    const sj_status st = engine_run_impl(err, e, jobs, k, on_done, user, mem);
    // device memory of the wave goes back to the pool on every path
    for (JobMem &m : mem) {
        dev_free(m.pts, e->st);
        dev_free(m.region, e->st);
        dev_free(m.out2, e->st);
    }
    if (cudaStreamSynchronize(e->st) != cudaSuccess) cudaGetLastError();
    return st;
}

void engine_tune_reset() {
    std::lock_guard<std::mutex> lk(g_wave_mu);
    g_wave_tuned.clear();
}

}  // namespace sj
