// index.cu -- grid index build (Section IV-B and IV-C).
//
// Steps, all on the device of the stream:
//   1. bounds: per-dimension min and max of the points (one host read-back,
//      the only synchronisation of the build); the host derives
//      g_min = min - eps, g_max = max + eps, the cell side w = eps (1 + 2^-16),
//      |g_j| = floor((g_max_j - g_min_j) / w) + 1 and the FP32 margin.
//   2. cell ids: c_j = floor((x_j - g_min_j) * (1 / w)) and the linear id
//      sum_j c_j * prod_{k<j} |g_k| (dimension 1 fastest), FP64.
//   3. sort by cell: a counting sort through a table over all grid cells
//      when the grid is small (the table then doubles as the dense lookup),
//      else an LSD radix sort.  The sorted point ids are the array A.
//   4. run-length compaction: B (sorted ids of the non-empty cells) and G
//      (start of each cell's range in A; cell h holds A[G[h] .. G[h+1])).
//   5. cell coordinates of every non-empty cell and the occupancy bitmaps
//      M_j (bit c of M_j set when some point has coordinate c in dim j).
//   6. cell-ordered point records: FP32 y_j = fl32(x_j - g_min_j) followed by
//      the point id (16 or 32 bytes per point, TMA/bulk-copy friendly), and
//      on demand the FP64 coordinates with the id.
//   7. work items (cell h, query block b): one per 32 points of each cell.
// Arrays whose length depends on |G| are allocated at their upper bound
// (|G| <= n), so no count has to come back to the host.
#include <cmath>
#include <cstring>

#include "grid_dev.cuh"

namespace sj {

namespace {

constexpr int kThreads = 256;

// minmax[2j] = min over points of x_j (order key), minmax[2j+1] = max.
// flag[0] |= 1 when a coordinate is NaN or infinite.
// Per-dimension min / max (order keys) and the non-finite flag: each block
// reduces its share in shared memory, then merges it with one atomic per
// bound.  MAXD: kMaxDim, or kMaxPointDim for the points of more dimensions.
template <int MAXD = kMaxDim>
__global__ void __launch_bounds__(kThreads) bounds_kernel(const double *__restrict__ pts,
                                                          uint64_t n, int d,
                                                          unsigned long long *minmax,
                                                          uint32_t *flag) {
    __shared__ unsigned long long s_mm[2 * MAXD];
    __shared__ uint32_t s_flag;
    if (threadIdx.x < 2 * MAXD) s_mm[threadIdx.x] = (threadIdx.x & 1) ? 0ULL : ~0ULL;
    if (threadIdx.x == 0) s_flag = 0u;
    __syncthreads();
    bounds_accumulate<MAXD>(pts, n, d, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (uint64_t)gridDim.x * blockDim.x, s_mm, &s_flag);
    __syncthreads();
    if (threadIdx.x < 2 * d) {
        if (threadIdx.x & 1)
            atomicMax(&minmax[threadIdx.x], s_mm[threadIdx.x]);
        else
            atomicMin(&minmax[threadIdx.x], s_mm[threadIdx.x]);
    }
    if (threadIdx.x == 0 && s_flag) atomicOr(flag, s_flag);
}

__global__ void init_minmax_kernel(unsigned long long *minmax, int d, uint32_t *flag) {
    int j = threadIdx.x;
    if (j < d) { minmax[2 * j] = ~0ULL; minmax[2 * j + 1] = 0ULL; }
    if (j == 0) *flag = 0;
}

// Linear cell id of each point; with a dense count table also the point's
// rank inside its cell.
__global__ void __launch_bounds__(kThreads) cell_kernel(const double *__restrict__ pts, uint64_t n,
                                                        CellParams cp, uint64_t *__restrict__ key,
                                                        uint32_t *__restrict__ val,
                                                        uint32_t *__restrict__ count) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t id = linear_cell(pts + i * cp.d, cp);
    key[i] = id;
    if (count)
        val[i] = atomicAdd(&count[id], 1u);
    else
        val[i] = (uint32_t)i;
}

// Linear cell id of each point, its rank inside its cell (dense count
// table) and its FP32 record in point order (tmp, rs floats per point):
// the offset x_j - g_min_j is computed once for the cell coordinate and
// the record coordinate.
__global__ void __launch_bounds__(kThreads) cell_rec_kernel(const double *__restrict__ pts,
                                                            uint64_t n, CellParams cp, int rs,
                                                            uint64_t *__restrict__ key,
                                                            uint32_t *__restrict__ val,
                                                            uint32_t *__restrict__ count,
                                                            float *__restrict__ tmp) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = pts + i * cp.d;
    float r[kMaxDim + 4];
    uint64_t id = 0;
#pragma unroll
    for (int j = 0; j < kMaxDim + 4; ++j) r[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
        if (j < cp.d) {
            const double a = __dsub_rn(p[j], cp.gmin[j]);
            const int64_t c = cell_of_offset(a, j, cp);
            id += (uint64_t)c * cp.stride[j];
            r[j] = rec_coord(a, c, cp);
        }
    }
#pragma unroll
    for (int j = 0; j <= kMaxDim; ++j)
        if (j == cp.d) r[j] = __uint_as_float((uint32_t)i);
    float4 *o = reinterpret_cast<float4 *>(tmp + i * rs);
#pragma unroll
    for (int v = 0; v < (kMaxDim + 4) / 4; ++v)
        if (4 * v < rs) o[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    key[i] = id;
    val[i] = atomicAdd(&count[id], 1u);
}

// Counting-sort scatter with the FP32 records: A[lut[id] + rank] = i, the
// sorted key and the point's record (rs floats, a multiple of 4) alongside.
__global__ void __launch_bounds__(kThreads) scatter_rec_kernel(const uint64_t *__restrict__ key,
                                                               const uint32_t *__restrict__ rank,
                                                               const uint32_t *__restrict__ lut,
                                                               uint64_t n, const float *__restrict__ tmp,
                                                               int rs, uint32_t *__restrict__ A,
                                                               uint64_t *__restrict__ skey,
                                                               float *__restrict__ rec) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t id = key[i];
    const uint64_t pos = lut[id] + rank[i];
    A[pos] = (uint32_t)i;
    skey[pos] = id;
    const float4 *src = reinterpret_cast<const float4 *>(tmp + i * rs);
    float4 *dst = reinterpret_cast<float4 *>(rec + pos * rs);
    float4 r[(kMaxDim + 4) / 4];
#pragma unroll
    for (int v = 0; v < (kMaxDim + 4) / 4; ++v)
        if (4 * v < rs) r[v] = src[v];
#pragma unroll
    for (int v = 0; v < (kMaxDim + 4) / 4; ++v)
        if (4 * v < rs) dst[v] = r[v];
}

// Counting-sort scatter: A[lut[id] + rank] = i, sorted key alongside.
__global__ void __launch_bounds__(kThreads) scatter_kernel(const uint64_t *__restrict__ key,
                                                           const uint32_t *__restrict__ rank,
                                                           const uint32_t *__restrict__ lut,
                                                           uint64_t n, uint32_t *__restrict__ A,
                                                           uint64_t *__restrict__ skey) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t id = key[i];
    uint32_t pos = lut[id] + rank[i];
    A[pos] = (uint32_t)i;
    skey[pos] = id;
}

__global__ void __launch_bounds__(kThreads) head_kernel(const uint64_t *__restrict__ skey,
                                                        uint64_t n, uint32_t *__restrict__ head) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    head[k] = (k == 0 || skey[k] != skey[k - 1]) ? 1u : 0u;
}

// head[] holds the exclusive scan of the head flags; a position k starts a
// cell when the scan steps at k.
__global__ void __launch_bounds__(kThreads) rle_kernel(const uint64_t *__restrict__ skey,
                                                       const uint32_t *__restrict__ hscan, uint64_t n,
                                                       const uint32_t *__restrict__ n_cells,
                                                       uint64_t *__restrict__ B,
                                                       uint32_t *__restrict__ G) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    bool is_head = (k == 0) || (skey[k] != skey[k - 1]);
    if (is_head) {
        uint32_t h = hscan[k];
        B[h] = skey[k];
        G[h] = (uint32_t)k;
    }
    if (k == 0) G[*n_cells] = (uint32_t)n;
}

// Cell coordinates and M_j of every non-empty cell (cells_block), grid-stride
// over the |G| cells counted on the device.
template <bool FROM_KEY>
__global__ void __launch_bounds__(kThreads) cells_kernel(const double *__restrict__ pts,
                                                         const uint32_t *__restrict__ A,
                                                         const uint32_t *__restrict__ G,
                                                         const uint64_t *__restrict__ B,
                                                         const uint32_t *__restrict__ n_cells,
                                                         CellParams cp, uint32_t mwords,
                                                         int32_t *__restrict__ cc,
                                                         uint32_t *__restrict__ M) {
    __shared__ uint32_t sm[kCellsSmemWords];
    cells_block<FROM_KEY>(pts, A, G, B, *n_cells, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                          (uint64_t)gridDim.x * blockDim.x, cp, mwords, cc, M, sm);
}

// FP32 record: y_j = fl32(x_j - g_min_j) for j < d, then the point id.
__global__ void __launch_bounds__(kThreads) rec32_kernel(const double *__restrict__ pts,
                                                         const uint32_t *__restrict__ A, uint64_t n,
                                                         CellParams cp, int rs,
                                                         float *__restrict__ rec) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    write_rec32(pts, A, k, cp, rs, rec);
}

__global__ void __launch_bounds__(kThreads) rec64_kernel(const double *__restrict__ pts,
                                                         const uint32_t *__restrict__ A, uint64_t n,
                                                         int d, int rs, double *__restrict__ rec) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    write_rec64(pts, A, k, d, rs, rec);
}

__global__ void __launch_bounds__(kThreads) item_count_kernel(const uint32_t *__restrict__ G,
                                                              const uint32_t *__restrict__ n_cells,
                                                              uint64_t cap,
                                                              uint32_t *__restrict__ cnt) {
    uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= cap) return;
    uint32_t nc = *n_cells;
    cnt[h] = h < nc ? (G[h + 1] - G[h] + kQueryBlock - 1) / kQueryBlock : 0u;
}

__global__ void __launch_bounds__(kThreads) item_fill_kernel(const uint32_t *__restrict__ G,
                                                             const uint32_t *__restrict__ n_cells,
                                                             const uint32_t *__restrict__ off,
                                                             uint2 *__restrict__ items) {
    uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= *n_cells) return;
    uint32_t nb = (G[h + 1] - G[h] + kQueryBlock - 1) / kQueryBlock;
    uint32_t o = off[h];
    for (uint32_t b = 0; b < nb; ++b) items[o + b] = make_uint2((uint32_t)h, b);
}

// Coordinate-tuple order (grids of 2^63 or more cells).  The points are
// sorted by one group of dimensions at a time, dimension 1 first, with the
// stable radix sort; a group packs the cell coordinates of its dimensions
// into one 64-bit key (higher dimensions in higher bits).
struct TupleGroup {
    int j0, j1;                    // dimensions [j0, j1)
    int shift[kMaxDim];            // bit position of c_j in the key
};

__global__ void __launch_bounds__(kThreads) iota_kernel(uint32_t *__restrict__ v, uint64_t n) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kThreads) tuple_key_kernel(const double *__restrict__ pts,
                                                             const uint32_t *__restrict__ val,
                                                             uint64_t n, CellParams cp, TupleGroup tg,
                                                             uint64_t *__restrict__ key) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *p = pts + (uint64_t)val[k] * cp.d;
    uint64_t y = 0;
    for (int j = tg.j0; j < tg.j1; ++j) y |= (uint64_t)cell_coord(p, j, cp) << tg.shift[j];
    key[k] = y;
}

// head[k] = 1 where the cell of the point at sorted position k differs from
// the previous one.
__global__ void __launch_bounds__(kThreads) tuple_head_kernel(const double *__restrict__ pts,
                                                              const uint32_t *__restrict__ A,
                                                              uint64_t n, CellParams cp,
                                                              uint32_t *__restrict__ head) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t h = 1;
    if (k > 0) {
        const double *p = pts + (uint64_t)A[k] * cp.d, *q = pts + (uint64_t)A[k - 1] * cp.d;
        h = 0;
        for (int j = 0; j < cp.d; ++j) h |= cell_coord(p, j, cp) != cell_coord(q, j, cp);
    }
    head[k] = h;
}

// G from the exclusive scan of the head flags (no B: there are no linear ids).
__global__ void __launch_bounds__(kThreads) tuple_rle_kernel(const uint32_t *__restrict__ hscan,
                                                             uint64_t n,
                                                             const uint32_t *__restrict__ n_cells,
                                                             uint32_t *__restrict__ G) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t next = k + 1 < n ? hscan[k + 1] : *n_cells;
    if (next != hscan[k]) G[hscan[k]] = (uint32_t)k;
    if (k == 0) G[*n_cells] = (uint32_t)n;
}

// High-dimensional path (more than kMaxDim dimensions) ---------------------

struct DimVals {
    double v[kMaxPointDim];
};

// proj[i][t] = x_i[gdim[t]]: the grid dimensions of every point.
struct GridDims {
    int v[kMaxDim];
};

__global__ void __launch_bounds__(kThreads) project_kernel(const double *__restrict__ pts,
                                                           uint64_t n, int d, int k, GridDims gd,
                                                           double *__restrict__ proj) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int t = 0; t < k; ++t) proj[i * k + t] = pts[i * d + gd.v[t]];
}

// Cell-ordered records of all d coordinates: fl32(x_j - fmin_j), then the id.
__global__ void __launch_bounds__(kThreads) recd32_kernel(const double *__restrict__ pts,
                                                          const uint32_t *__restrict__ A,
                                                          uint64_t n, int d, DimVals fmin, int rs,
                                                          float *__restrict__ rec) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t i = A[k];
    const double *p = pts + (uint64_t)i * d;
    float *r = rec + k * rs;
    for (int j = 0; j < d; ++j) r[j] = __double2float_rn(__dsub_rn(p[j], fmin.v[j]));
    r[d] = __uint_as_float(i);
    for (int j = d + 1; j < rs; ++j) r[j] = 0.0f;
}

inline unsigned grid_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Blocks of a grid-stride kernel over n elements: enough for full occupancy
// (eight blocks of kThreads per SM), fewer when n is small.
inline unsigned grid_stride_blocks(uint64_t n) {
    const uint64_t want = 8ull * (uint64_t)sm_count(-1);
    const uint64_t need = (n + kThreads - 1) / kThreads;
    return (unsigned)(need < want ? (need ? need : 1) : want);
}

}  // namespace

// Geometry of Section IV-B from the per-dimension bounds (order keys,
// mm[2j] = min, mm[2j+1] = max): g_min = min - eps, g_max = max + eps, cell
// side w = eps (1 + 2^-16), |g_j| = floor((g_max_j - g_min_j) / w) + 1,
// strides with dimension 1 fastest, and the FP32 margin.
sj_status geometry_from_bounds(Error &err, const unsigned long long *mm, int d, uint64_t n,
                               double eps, int frame_mode, Geometry &g) {
    g = Geometry();
    g.d = d;
    g.n = n;
    g.eps = eps;
    g.E2 = eps * eps;
    g.w = eps * (1.0 + std::ldexp(1.0, -16));
    double total = 1.0;
    for (int j = 0; j < d; ++j) {
        const double mn = from_order_key(mm[2 * j]), mx = from_order_key(mm[2 * j + 1]);
        g.gmin[j] = mn - eps;
        g.gmax[j] = mx + eps;
        const double cells = std::floor((g.gmax[j] - g.gmin[j]) / g.w) + 1.0;
        if (!(cells < 2147483648.0)) return fail(err, SJ_ERANGE, "a dimension needs 2^31 or more cells");
        g.ng[j] = (int64_t)cells;
        total *= cells;
    }
    if (total < 9.2e18) {
        uint64_t stride = 1;
        for (int j = 0; j < d; ++j) {
            g.stride[j] = stride;
            stride *= (uint64_t)g.ng[j];
        }
        g.grid_cells = stride;
    } else {
        // linear ids would not fit in 64 bits: cells are ordered by their
        // coordinate tuples instead (the same order)
        g.huge = 1;
        g.grid_cells = ~0ull;
    }
    fp32_margin(g, frame_mode);  // margin.cu
    return SJ_OK;
}

// True when p is 8-byte aligned device (or managed) memory of the current
// device, so that the index kernels may read it in place.
static bool device_array_here(const void *p) {
    if (reinterpret_cast<uintptr_t>(p) & 7u) return false;
    cudaPointerAttributes at;
    int dev = -1;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

void free_index(Index &ix, cudaStream_t s) {
    if (ix.pts_borrowed) {
        ix.pts = DevBuf();
        ix.pts_borrowed = 0;
    }
    DevBuf *all[] = {&ix.pts, &ix.rec32, &ix.rec64, &ix.A,          &ix.B,
                     &ix.G,   &ix.cc,    &ix.M,     &ix.lut,        &ix.items,
                     &ix.counts_dev,     &ix.ptsd,  &ix.recd32,     &ix.recd64, &ix.hmid_dev};
    for (DevBuf *b : all) dev_free(*b, s);
}

// Small device scratch for counts that the host may read later.
struct BuildScratch {
    DevBuf minmax, counts;  // counts: [0] flag, [1] n_cells, [2] n_items, [3] lut total
};

sj_status bounds_of(Error &err, const double *d_pts, uint64_t n, int d, cudaStream_t s,
                    unsigned long long *mm, bool *nonfinite) {
    DevBuf scratch;
    SJ_TRY(dev_alloc(err, scratch, (2 * kMaxDim) * sizeof(unsigned long long) + 64, s));
    unsigned long long *d_minmax = static_cast<unsigned long long *>(scratch.p);
    uint32_t *d_flag = reinterpret_cast<uint32_t *>(d_minmax + 2 * kMaxDim);
    init_minmax_kernel<<<1, 32, 0, s>>>(d_minmax, d, d_flag); note_launch();
    bounds_kernel<><<<grid_stride_blocks(n), kThreads, 0, s>>>(d_pts, n, d, d_minmax, d_flag); note_launch();
    unsigned long long h[2 * kMaxDim + 8];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_minmax, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(scratch, s);
    if (e != cudaSuccess) {
        set_cuda_error(err, e, "bounds", __FILE__, __LINE__);
        return err.st;
    }
    for (int k = 0; k < 2 * kMaxDim; ++k) mm[k] = h[k];
    *nonfinite = (reinterpret_cast<const uint32_t *>(h + 2 * kMaxDim)[0] & 1u) != 0;
    return SJ_OK;
}

// Index of points with more than kMaxDim dimensions: bounds of every
// dimension, the kHdGridDims dimensions with the most cells as the grid
// (built by build_index from the projected points), then the cell-ordered
// records of all coordinates and the margin of the difference-form filter.
static sj_status build_index_hd(Error &err, const double *pts_any, uint64_t n, int d, double eps,
                                int lookup_mode, cudaStream_t s, Index &ix) {
    ix = Index();
    ix.owner_stream = s;
    if (n >= (1ull << 32)) return fail(err, SJ_ERANGE, "n must be below 2^32");
    DevBuf full, proj, scratch;
    auto cleanup = [&]() { dev_free(full, s); dev_free(proj, s); dev_free(scratch, s); };
    sj_status st = SJ_OK;
#define SJ_HDT(expr) do { st = (expr); if (st != SJ_OK) { cleanup(); return st; } } while (0)
#define SJ_HDC(expr) do { cudaError_t e__ = (expr); if (e__ != cudaSuccess) { set_cuda_error(err, e__, #expr, __FILE__, __LINE__); cleanup(); return err.st; } } while (0)
    SJ_HDT(dev_alloc(err, full, n * d * sizeof(double), s));
    SJ_HDC(cudaMemcpyAsync(full.p, pts_any, n * d * sizeof(double), cudaMemcpyDefault, s));
    const double *pts = static_cast<const double *>(full.p);
    SJ_HDT(dev_alloc(err, scratch, (2 * kMaxPointDim) * sizeof(unsigned long long) + 64, s));
    unsigned long long *d_minmax = static_cast<unsigned long long *>(scratch.p);
    uint32_t *d_flag = reinterpret_cast<uint32_t *>(d_minmax + 2 * kMaxPointDim);
    init_minmax_kernel<<<1, 32, 0, s>>>(d_minmax, d, d_flag); note_launch();
    bounds_kernel<kMaxPointDim><<<grid_stride_blocks(n), kThreads, 0, s>>>(pts, n, d, d_minmax, d_flag);
    note_launch();
    SJ_HDC(cudaGetLastError());
    unsigned long long h[2 * kMaxPointDim + 8];
    SJ_HDC(cudaMemcpyAsync(h, d_minmax, sizeof(h), cudaMemcpyDeviceToHost, s));
    SJ_HDC(cudaStreamSynchronize(s));
    if (reinterpret_cast<const uint32_t *>(h + 2 * kMaxPointDim)[0] & 1u) {
        cleanup();
        return fail(err, SJ_EINVAL, "non-finite coordinate");
    }
    const double w = eps * (1.0 + std::ldexp(1.0, -16));
    double fmin[kMaxPointDim], fmax[kMaxPointDim], cells[kMaxPointDim];
    for (int j = 0; j < d; ++j) {
        fmin[j] = from_order_key(h[2 * j]) - eps;
        fmax[j] = from_order_key(h[2 * j + 1]) + eps;
        cells[j] = std::floor((fmax[j] - fmin[j]) / w) + 1.0;
    }
    // the grid: the kHdGridDims dimensions with the most cells, in order
    bool taken[kMaxPointDim] = {};
    for (int t = 0; t < kHdGridDims; ++t) {
        int best = -1;
        for (int j = 0; j < d; ++j)
            if (!taken[j] && (best < 0 || cells[j] > cells[best])) best = j;
        taken[best] = true;
    }
    GridDims gd;
    int k = 0;
    for (int j = 0; j < d; ++j)
        if (taken[j]) gd.v[k++] = j;
    unsigned long long mm[2 * kMaxDim];
    for (int t = 0; t < k; ++t) {
        mm[2 * t] = h[2 * gd.v[t]];
        mm[2 * t + 1] = h[2 * gd.v[t] + 1];
    }
    SJ_HDT(dev_alloc(err, proj, n * k * sizeof(double), s));
    project_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, n, d, k, gd, static_cast<double *>(proj.p));
    note_launch();
    SJ_HDC(cudaGetLastError());
    Index inner;
    st = build_index(err, static_cast<const double *>(proj.p), n, k, eps, lookup_mode, SJ_FRAME_GRID,
                     s, inner, mm);
    if (st != SJ_OK) {
        free_index(inner, s);
        cleanup();
        return st;
    }
    ix = inner;
    dev_free(proj, s);
    dev_free(scratch, s);
    ix.dfull = d;
    for (int t = 0; t < k; ++t) ix.gdim[t] = gd.v[t];
    for (int j = 0; j < d; ++j) {
        ix.fmin[j] = fmin[j];
        ix.fmax[j] = fmax[j];
    }
    ix.ptsd = full;
    full = DevBuf();
    ix.rsd32 = (d + 1 + 3) / 4 * 4;
    ix.rsd64 = (d + 1 + 1) / 2 * 2;
    DimVals fv;
    for (int j = 0; j < kMaxPointDim; ++j) fv.v[j] = j < d ? fmin[j] : 0.0;
    st = dev_alloc(err, ix.recd32, n * ix.rsd32 * sizeof(float), s);
    if (st != SJ_OK) { free_index(ix, s); return st; }
    recd32_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double *>(ix.ptsd.p),
                                                   static_cast<const uint32_t *>(ix.A.p), n, d, fv,
                                                   ix.rsd32, static_cast<float *>(ix.recd32.p));
    note_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(err, e, "recd32_kernel", __FILE__, __LINE__);
        free_index(ix, s);
        return err.st;
    }
    Geometry &g = ix.g;
    // the expanded-form sum (one fma per coordinate) while its band is
    // narrow (below 2^-10 E2, the rule of the frame choice), else the
    // difference form (two per coordinate, a band 10-100x narrower), else
    // the expanded form when only it has a margin (margin.cu)
    int grid[kMaxPointDim] = {};
    for (int t = 0; t < k; ++t) grid[gd.v[t]] = 1;
    float elo = -1.0f, ehi = 0.0f, dlo = -1.0f, dhi = 0.0f;
    const bool eok = fp32_margin_hd(d, eps, fmin, fmax, grid, &elo, &ehi, ix.hmid);
    const bool dok = fp32_margin_diff(d, eps, fmin, fmax, &dlo, &dhi);
    const double eband = (double)ehi - (elo > 0.0f ? (double)elo : 0.0);
    ix.hd_exp = (eok && (eband <= std::ldexp(g.E2, -10) || !dok)) ? 1 : 0;
    g.fp32_ok = (ix.hd_exp || dok) ? 1 : 0;
    g.lo32 = ix.hd_exp ? elo : dlo;
    g.hi32 = ix.hd_exp ? ehi : dhi;
    st = dev_alloc(err, ix.hmid_dev, sizeof(ix.hmid), s);
    if (st == SJ_OK && cudaMemcpyAsync(ix.hmid_dev.p, ix.hmid, sizeof(ix.hmid), cudaMemcpyHostToDevice, s) !=
                           cudaSuccess) {
        cudaGetLastError();
        st = fail(err, SJ_ECUDA, "copy of the high-dimensional origin failed");
    }
    if (st != SJ_OK) { free_index(ix, s); return st; }
    g.frame = SJ_FRAME_GRID;
    ix.bytes += ix.ptsd.bytes + ix.recd32.bytes;
#undef SJ_HDT
#undef SJ_HDC
    return SJ_OK;
}

sj_status build_index(Error &err, const double *pts_any, uint64_t n, int d, double eps,
                      int lookup_mode, int frame_mode, cudaStream_t s, Index &ix,
                      const unsigned long long *given_mm, const BuildOpts *opt) {
    if (d > kMaxDim && d <= kMaxPointDim && !given_mm && pts_any && n && eps > 0.0 &&
        std::isfinite(eps))
        return build_index_hd(err, pts_any, n, d, eps, lookup_mode, s, ix);
    ix = Index();
    ix.owner_stream = s;
    if (pts_any == nullptr || n == 0 || d < 1 || d > kMaxDim || !(eps > 0.0) || !std::isfinite(eps))
        return fail(err, SJ_EINVAL, "invalid argument (pts, n, d in [1,8], eps > 0 finite)");
    if (n >= (1ull << 32)) return fail(err, SJ_ERANGE, "n must be below 2^32");
    Geometry &g = ix.g;
    g.d = d;
    g.n = n;
    g.eps = eps;
    g.E2 = eps * eps;
    g.w = eps * (1.0 + std::ldexp(1.0, -16));

    // 1. points on the device: the caller's array when it may be borrowed,
    // else a copy the index owns
    if (opt && opt->borrow_pts && device_array_here(pts_any)) {
        ix.pts.p = const_cast<double *>(pts_any);
        ix.pts_borrowed = 1;
    } else {
        SJ_TRY(dev_alloc(err, ix.pts, n * d * sizeof(double), s));
        SJ_CUDA_TRY(cudaMemcpyAsync(ix.pts.p, pts_any, n * d * sizeof(double), cudaMemcpyDefault, s));
    }
    const double *pts = static_cast<const double *>(ix.pts.p);

    // bounds
    DevBuf scratch;
    SJ_TRY(dev_alloc(err, scratch, (2 * kMaxDim) * sizeof(unsigned long long) + 64, s));
    unsigned long long *d_minmax = static_cast<unsigned long long *>(scratch.p);
    uint32_t *d_counts = reinterpret_cast<uint32_t *>(d_minmax + 2 * kMaxDim);
    SJ_CUDA_TRY(cudaMemsetAsync(d_counts, 0, 64, s));
    unsigned long long h_mm[2 * kMaxDim + 8];
    if (given_mm) {
        // bounds given by the caller (a grid shared with another point set)
        for (int k = 0; k < 2 * kMaxDim; ++k) h_mm[k] = given_mm[k];
    } else {
        init_minmax_kernel<<<1, 32, 0, s>>>(d_minmax, d, d_counts); note_launch();
        bounds_kernel<><<<grid_stride_blocks(n), kThreads, 0, s>>>(pts, n, d, d_minmax, d_counts); note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        SJ_CUDA_TRY(cudaMemcpyAsync(h_mm, d_minmax, sizeof(h_mm), cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        const uint32_t *h_counts = reinterpret_cast<const uint32_t *>(h_mm + 2 * kMaxDim);
        if (h_counts[0] & 1u) { dev_free(scratch, s); return fail(err, SJ_EINVAL, "non-finite coordinate"); }
    }

    // geometry (Section IV-B)
    {
        const sj_status gst = geometry_from_bounds(err, h_mm, d, n, eps, frame_mode, g);
        if (gst != SJ_OK) { dev_free(scratch, s); return gst; }
    }

    // 2-3. cell ids and the sort by cell
    uint64_t dense_limit = (uint64_t)16 * n;
    if (dense_limit < (1ull << 25)) dense_limit = 1ull << 25;
    const bool tuple = g.huge || lookup_mode == SJ_LOOKUP_COORDS;
    bool dense = !tuple && ((lookup_mode == SJ_LOOKUP_DENSE && g.grid_cells < (1ull << 32) - 1) ||
                            (lookup_mode == SJ_LOOKUP_AUTO && g.grid_cells <= dense_limit));
    ix.dense = dense ? 1 : 0;
    ix.tuple = tuple ? 1 : 0;

    const CellParams cp = cell_params(g);

    ix.rs32 = (d + 1 + 3) / 4 * 4;
    ix.rs64 = (d + 1 + 1) / 2 * 2;
    DevBuf key, val, skey_buf, head, rtmp;
    auto cleanup = [&]() {
        dev_free(key, s); dev_free(val, s); dev_free(skey_buf, s); dev_free(head, s);
        dev_free(rtmp, s); dev_free(scratch, s);
    };
    sj_status st = SJ_OK;
#define SJ_B(expr) do { st = (expr); if (st != SJ_OK) { cleanup(); return st; } } while (0)
#define SJ_BC(expr) do { cudaError_t e__ = (expr); if (e__ != cudaSuccess) { set_cuda_error(err, e__, #expr, __FILE__, __LINE__); cleanup(); return err.st; } } while (0)
    SJ_B(dev_alloc(err, key, n * sizeof(uint64_t), s));
    SJ_B(dev_alloc(err, val, n * sizeof(uint32_t), s));
    SJ_B(dev_alloc(err, ix.A, n * sizeof(uint32_t), s));
    uint64_t *skey = nullptr;
    if (dense) {
        SJ_B(dev_alloc(err, ix.lut, (g.grid_cells + 1) * sizeof(uint32_t), s));
        uint32_t *lut = static_cast<uint32_t *>(ix.lut.p);
        SJ_BC(cudaMemsetAsync(lut, 0, (g.grid_cells + 1) * sizeof(uint32_t), s));
        // the FP32 records are written in point order by the cell pass and
        // moved to cell order by the scatter
        SJ_B(dev_alloc(err, rtmp, n * ix.rs32 * sizeof(float), s));
        SJ_B(dev_alloc(err, ix.rec32, n * ix.rs32 * sizeof(float), s));
        cell_rec_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, n, cp, ix.rs32, static_cast<uint64_t *>(key.p),
                                                         static_cast<uint32_t *>(val.p), lut,
                                                         static_cast<float *>(rtmp.p)); note_launch();
        SJ_BC(cudaGetLastError());
        SJ_B(exclusive_scan_u32(err, lut, lut, g.grid_cells + 1, d_counts + 3, s));
        SJ_B(dev_alloc(err, skey_buf, n * sizeof(uint64_t), s));
        skey = static_cast<uint64_t *>(skey_buf.p);
        scatter_rec_kernel<<<grid_for(n), kThreads, 0, s>>>(
            static_cast<uint64_t *>(key.p), static_cast<uint32_t *>(val.p), lut, n,
            static_cast<const float *>(rtmp.p), ix.rs32, static_cast<uint32_t *>(ix.A.p), skey,
            static_cast<float *>(ix.rec32.p)); note_launch();
        SJ_BC(cudaGetLastError());
        dev_free(rtmp, s);
    } else if (tuple) {
        uint32_t *v = static_cast<uint32_t *>(val.p);
        iota_kernel<<<grid_for(n), kThreads, 0, s>>>(v, n); note_launch();
        SJ_BC(cudaGetLastError());
        for (int j0 = 0; j0 < d;) {
            TupleGroup tg;
            std::memset(&tg, 0, sizeof(tg));
            tg.j0 = j0;
            int bits = 0, j = j0;
            while (j < d) {
                int bj = 1;
                while (bj < 31 && ((uint64_t)(g.ng[j] - 1) >> bj)) ++bj;
                if (bits + bj > 64) break;
                tg.shift[j] = bits;
                bits += bj;
                ++j;
            }
            tg.j1 = j;
            tuple_key_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, v, n, cp, tg,
                                                              static_cast<uint64_t *>(key.p)); note_launch();
            SJ_BC(cudaGetLastError());
            SJ_B(radix_sort_pairs(err, static_cast<uint64_t *>(key.p), v, n, bits, s));
            j0 = j;
        }
        SJ_BC(cudaMemcpyAsync(ix.A.p, val.p, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    } else {
        cell_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, n, cp, static_cast<uint64_t *>(key.p),
                                                     static_cast<uint32_t *>(val.p), nullptr); note_launch();
        SJ_BC(cudaGetLastError());
        int bits = 0;
        while (bits < 64 && (g.grid_cells - 1) >> bits) ++bits;
        SJ_B(radix_sort_pairs(err, static_cast<uint64_t *>(key.p), static_cast<uint32_t *>(val.p),
                              n, bits, s));
        SJ_BC(cudaMemcpyAsync(ix.A.p, val.p, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        skey = static_cast<uint64_t *>(key.p);
    }

    // 4. B and G
    SJ_B(dev_alloc(err, head, n * sizeof(uint32_t), s));
    uint32_t *hs = static_cast<uint32_t *>(head.p);
    if (tuple)
        tuple_head_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, static_cast<const uint32_t *>(ix.A.p),
                                                           n, cp, hs);
    else
        head_kernel<<<grid_for(n), kThreads, 0, s>>>(skey, n, hs);
    note_launch();
    SJ_BC(cudaGetLastError());
    SJ_B(exclusive_scan_u32(err, hs, hs, n, d_counts + 1, s));
    SJ_B(dev_alloc(err, ix.G, (n + 1) * sizeof(uint32_t), s));
    // the scan total counts heads before position n = |G|
    if (tuple) {
        tuple_rle_kernel<<<grid_for(n), kThreads, 0, s>>>(hs, n, d_counts + 1,
                                                          static_cast<uint32_t *>(ix.G.p));
    } else {
        SJ_B(dev_alloc(err, ix.B, n * sizeof(uint64_t), s));
        rle_kernel<<<grid_for(n), kThreads, 0, s>>>(skey, hs, n, d_counts + 1,
                                                     static_cast<uint64_t *>(ix.B.p),
                                                     static_cast<uint32_t *>(ix.G.p));
    }
    note_launch();
    SJ_BC(cudaGetLastError());
    if (opt && opt->h_counts && opt->ev_counts) {
        SJ_BC(cudaMemcpyAsync(opt->h_counts, d_counts, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SJ_BC(cudaEventRecord(opt->ev_counts, s));
        ix.early_counts = opt->h_counts;
        ix.early_ev = opt->ev_counts;
    }

    // 5. cell coordinates and M_j
    uint64_t maxng = 1;
    for (int j = 0; j < d; ++j) maxng = (uint64_t)g.ng[j] > maxng ? (uint64_t)g.ng[j] : maxng;
    ix.mwords = (uint32_t)((maxng + 31) / 32);
    SJ_B(dev_alloc(err, ix.cc, n * d * sizeof(int32_t), s));
    SJ_B(dev_alloc(err, ix.M, (uint64_t)d * ix.mwords * sizeof(uint32_t), s));
    SJ_BC(cudaMemsetAsync(ix.M.p, 0, (uint64_t)d * ix.mwords * sizeof(uint32_t), s));
    if (tuple)
        cells_kernel<false><<<grid_stride_blocks(n), kThreads, 0, s>>>(
            pts, static_cast<const uint32_t *>(ix.A.p), static_cast<const uint32_t *>(ix.G.p), nullptr,
            d_counts + 1, cp, ix.mwords, static_cast<int32_t *>(ix.cc.p), static_cast<uint32_t *>(ix.M.p));
    else
        cells_kernel<true><<<grid_stride_blocks(n), kThreads, 0, s>>>(
            pts, nullptr, nullptr, static_cast<const uint64_t *>(ix.B.p), d_counts + 1, cp, ix.mwords,
            static_cast<int32_t *>(ix.cc.p), static_cast<uint32_t *>(ix.M.p));
    note_launch();
    SJ_BC(cudaGetLastError());

    // 6. FP32 records (already in place on the dense path)
    if (!ix.rec32.p) {
        SJ_B(dev_alloc(err, ix.rec32, n * ix.rs32 * sizeof(float), s));
        rec32_kernel<<<grid_for(n), kThreads, 0, s>>>(pts, static_cast<uint32_t *>(ix.A.p), n, cp,
                                                      ix.rs32, static_cast<float *>(ix.rec32.p)); note_launch();
        SJ_BC(cudaGetLastError());
    }

    // 7. work items
    uint32_t *icnt = static_cast<uint32_t *>(val.p);  // reuse: n entries
    item_count_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint32_t *>(ix.G.p), d_counts + 1, n,
                                                       icnt); note_launch();
    SJ_BC(cudaGetLastError());
    SJ_B(exclusive_scan_u32(err, icnt, icnt, n, d_counts + 2, s));
    SJ_B(dev_alloc(err, ix.items, n * sizeof(uint2), s));
    item_fill_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint32_t *>(ix.G.p), d_counts + 1,
                                                      icnt, static_cast<uint2 *>(ix.items.p)); note_launch();
    SJ_BC(cudaGetLastError());

    dev_free(key, s);
    dev_free(val, s);
    dev_free(skey_buf, s);
    dev_free(head, s);
    // keep the counters (n_cells, n_items) on the device inside the index
    ix.counts_dev = scratch;
    ix.bytes = ix.pts.bytes + ix.rec32.bytes + ix.A.bytes + ix.B.bytes + ix.G.bytes + ix.cc.bytes +
               ix.M.bytes + ix.lut.bytes + ix.items.bytes + scratch.bytes;
#undef SJ_B
#undef SJ_BC
    return SJ_OK;
}

// Builds the FP64 records when a FP64-mode join first needs them.
sj_status ensure_rec64(Error &err, Index &ix, cudaStream_t s) {
    if (ix.dfull > kMaxDim) {
        if (ix.recd64.p) return SJ_OK;
        const uint64_t n = ix.g.n;
        SJ_TRY(dev_alloc(err, ix.recd64, n * ix.rsd64 * sizeof(double), s));
        rec64_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double *>(ix.ptsd.p),
                                                      static_cast<const uint32_t *>(ix.A.p), n,
                                                      ix.dfull, ix.rsd64,
                                                      static_cast<double *>(ix.recd64.p)); note_launch();
        SJ_CUDA_TRY(cudaGetLastError());
        ix.bytes += ix.recd64.bytes;
        return SJ_OK;
    }
    if (ix.rec64.p) return SJ_OK;
    const uint64_t n = ix.g.n;
    SJ_TRY(dev_alloc(err, ix.rec64, n * ix.rs64 * sizeof(double), s));
    rec64_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double *>(ix.pts.p),
                                                  static_cast<const uint32_t *>(ix.A.p), n, ix.g.d,
                                                  ix.rs64, static_cast<double *>(ix.rec64.p)); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    ix.bytes += ix.rec64.bytes;
    return SJ_OK;
}

// Reads |G| and the number of work items back to the host (synchronises s).
sj_status read_counts(Error &err, Index &ix, cudaStream_t s) {
    if (ix.counts_read) return SJ_OK;
    uint32_t h[4];
    const uint32_t *d_counts = reinterpret_cast<const uint32_t *>(
        static_cast<unsigned long long *>(ix.counts_dev.p) + 2 * kMaxDim);
    SJ_CUDA_TRY(cudaMemcpyAsync(h, d_counts, sizeof(h), cudaMemcpyDeviceToHost, s));
    SJ_CUDA_TRY(cudaStreamSynchronize(s));
    ix.n_cells = h[1];
    ix.n_items = h[2];
    ix.counts_read = 1;
    return SJ_OK;
}

const uint32_t *n_items_dev(const Index &ix) {
    return reinterpret_cast<const uint32_t *>(static_cast<unsigned long long *>(ix.counts_dev.p) +
                                              2 * kMaxDim) + 2;
}

// Index build for callers that cannot allocate device memory: the same
// kernels as build_index, with every array carved from `region` (a device
// address, region_bytes long) and the points read in place from d_pts (a
// device pointer that must stay valid while the index is used).  Dense
// lookup table only (grid_cells <= max_grid_cells, else SJ_ERANGE); nothing
// is allocated and the returned Index owns nothing (never pass it to
// free_index).
sj_status build_index_static(Error &err, const double *d_pts, uint64_t n, int d, double eps,
                             unsigned char *region, size_t region_bytes, uint64_t max_grid_cells,
                             cudaStream_t s, Index &ix) {
    ix = Index();
    ix.owner_stream = s;
    if (d_pts == nullptr || n == 0 || d < 1 || d > kMaxDim || !(eps > 0.0) || !std::isfinite(eps))
        return fail(err, SJ_EINVAL, "invalid argument (pts, n, d in [1,8], eps > 0 finite)");
    size_t off = 0;
    bool exhausted = false;
    auto take = [&](DevBuf &b, size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        if (off + bytes > region_bytes) { exhausted = true; return; }
        b.p = region + off;
        b.bytes = bytes;
        off += bytes;
    };
    Geometry &g = ix.g;
    g.d = d;
    g.n = n;
    g.eps = eps;
    g.E2 = eps * eps;
    g.w = eps * (1.0 + std::ldexp(1.0, -16));
    ix.pts.p = const_cast<double *>(d_pts);
    ix.pts.bytes = n * d * sizeof(double);

    take(ix.counts_dev, (2 * kMaxDim) * sizeof(unsigned long long) + 64);
    if (exhausted) return fail(err, SJ_ERANGE, "static scratch exhausted");
    unsigned long long *d_minmax = static_cast<unsigned long long *>(ix.counts_dev.p);
    uint32_t *d_counts = reinterpret_cast<uint32_t *>(d_minmax + 2 * kMaxDim);
    SJ_CUDA_TRY(cudaMemsetAsync(d_counts, 0, 64, s));
    init_minmax_kernel<<<1, 32, 0, s>>>(d_minmax, d, d_counts); note_launch();
    bounds_kernel<><<<grid_stride_blocks(n), kThreads, 0, s>>>(d_pts, n, d, d_minmax, d_counts); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    unsigned long long h_mm[2 * kMaxDim + 8];
    SJ_CUDA_TRY(cudaMemcpyAsync(h_mm, d_minmax, sizeof(h_mm), cudaMemcpyDeviceToHost, s));
    SJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (reinterpret_cast<const uint32_t *>(h_mm + 2 * kMaxDim)[0] & 1u)
        return fail(err, SJ_EINVAL, "non-finite coordinate");
    uint64_t stride = 1;
    double total = 1.0;
    for (int j = 0; j < d; ++j) {
        g.gmin[j] = from_order_key(h_mm[2 * j]) - eps;
        g.gmax[j] = from_order_key(h_mm[2 * j + 1]) + eps;
        const double cells = std::floor((g.gmax[j] - g.gmin[j]) / g.w) + 1.0;
        total *= cells;
        if (!(cells < 2147483648.0) || !(total <= (double)max_grid_cells))
            return fail(err, SJ_ERANGE, "grid larger than the static lookup table allows");
        g.ng[j] = (int64_t)cells;
        g.stride[j] = stride;
        stride *= (uint64_t)g.ng[j];
    }
    g.grid_cells = stride;
    fp32_margin(g, SJ_FRAME_AUTO);
    ix.dense = 1;

    const CellParams cp = cell_params(g);
    uint64_t maxng = 1;
    for (int j = 0; j < d; ++j) maxng = (uint64_t)g.ng[j] > maxng ? (uint64_t)g.ng[j] : maxng;
    ix.mwords = (uint32_t)((maxng + 31) / 32);
    ix.rs32 = (d + 1 + 3) / 4 * 4;
    ix.rs64 = (d + 1 + 1) / 2 * 2;
    DevBuf key, rank, skey, head, sums;
    take(ix.lut, (g.grid_cells + 1) * sizeof(uint32_t));
    take(key, n * sizeof(uint64_t));
    take(rank, n * sizeof(uint32_t));
    take(ix.A, n * sizeof(uint32_t));
    take(skey, n * sizeof(uint64_t));
    take(head, n * sizeof(uint32_t));
    take(ix.B, n * sizeof(uint64_t));
    take(ix.G, (n + 1) * sizeof(uint32_t));
    take(ix.cc, n * d * sizeof(int32_t));
    take(ix.M, (uint64_t)d * ix.mwords * sizeof(uint32_t));
    take(ix.rec32, n * ix.rs32 * sizeof(float));
    take(ix.items, n * sizeof(uint2));
    const uint64_t scan_max = (g.grid_cells + 1) > n ? (g.grid_cells + 1) : n;
    take(sums, scan_sums_needed(scan_max) * sizeof(uint32_t));
    if (!g.fp32_ok) take(ix.rec64, n * ix.rs64 * sizeof(double));
    if (exhausted) return fail(err, SJ_ERANGE, "static scratch exhausted");
    uint32_t *lut = static_cast<uint32_t *>(ix.lut.p);
    uint32_t *ps = static_cast<uint32_t *>(sums.p);
    const size_t ps_cap = sums.bytes / sizeof(uint32_t);

    // the region keeps the previous call's contents: clear what accumulates
    SJ_CUDA_TRY(cudaMemsetAsync(lut, 0, (g.grid_cells + 1) * sizeof(uint32_t), s));
    SJ_CUDA_TRY(cudaMemsetAsync(ix.M.p, 0, ix.M.bytes, s));
    cell_kernel<<<grid_for(n), kThreads, 0, s>>>(d_pts, n, cp, static_cast<uint64_t *>(key.p),
                                                 static_cast<uint32_t *>(rank.p), lut); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    SJ_TRY(exclusive_scan_u32_scratch(err, lut, lut, g.grid_cells + 1, d_counts + 3, ps, ps_cap, s));
    scatter_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint64_t *>(key.p),
                                                    static_cast<uint32_t *>(rank.p), lut, n,
                                                    static_cast<uint32_t *>(ix.A.p),
                                                    static_cast<uint64_t *>(skey.p)); note_launch();
    uint32_t *hs = static_cast<uint32_t *>(head.p);
    head_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint64_t *>(skey.p), n, hs); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    SJ_TRY(exclusive_scan_u32_scratch(err, hs, hs, n, d_counts + 1, ps, ps_cap, s));
    rle_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint64_t *>(skey.p), hs, n, d_counts + 1,
                                                 static_cast<uint64_t *>(ix.B.p),
                                                 static_cast<uint32_t *>(ix.G.p)); note_launch();
    cells_kernel<true><<<grid_stride_blocks(n), kThreads, 0, s>>>(
        d_pts, nullptr, nullptr, static_cast<const uint64_t *>(ix.B.p), d_counts + 1, cp, ix.mwords,
        static_cast<int32_t *>(ix.cc.p), static_cast<uint32_t *>(ix.M.p)); note_launch();
    rec32_kernel<<<grid_for(n), kThreads, 0, s>>>(d_pts, static_cast<uint32_t *>(ix.A.p), n, cp,
                                                  ix.rs32, static_cast<float *>(ix.rec32.p)); note_launch();
    if (ix.rec64.p) {
        rec64_kernel<<<grid_for(n), kThreads, 0, s>>>(d_pts, static_cast<const uint32_t *>(ix.A.p), n, d,
                                                      ix.rs64, static_cast<double *>(ix.rec64.p)); note_launch();
    }
    SJ_CUDA_TRY(cudaGetLastError());
    uint32_t *icnt = static_cast<uint32_t *>(rank.p);   // ranks are consumed by now
    item_count_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint32_t *>(ix.G.p), d_counts + 1,
                                                       n, icnt); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    SJ_TRY(exclusive_scan_u32_scratch(err, icnt, icnt, n, d_counts + 2, ps, ps_cap, s));
    item_fill_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<uint32_t *>(ix.G.p), d_counts + 1,
                                                      icnt, static_cast<uint2 *>(ix.items.p)); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    ix.bytes = off;
    return SJ_OK;
}

}  // namespace sj
