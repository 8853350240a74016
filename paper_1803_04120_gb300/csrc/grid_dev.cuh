// grid_dev.cuh -- device helpers of the grid index (Section IV-B) shared by
// the single-join build (index.cu) and the batched multi-join build
// (engine.cu).
#pragma once

#include <cstring>

#include "sj_internal.cuh"

namespace sj {

// Order-preserving map of a double onto an unsigned integer, so that min and
// max reduce with integer atomics.
__device__ __forceinline__ unsigned long long order_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}

__host__ __device__ inline double from_order_key(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ULL) ? (k & 0x7fffffffffffffffULL) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof(x));
    return x;
#endif
}

// What the cell-id kernels need of the geometry.
struct CellParams {
    int d;
    int frame;                 // sj_frame of the FP32 records
    double gmin[kMaxDim];
    double inv_w;
    double w;
    int64_t ng[kMaxDim];
    uint64_t stride[kMaxDim];
};

inline CellParams cell_params(const Geometry &g) {
    CellParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.d = g.d;
    cp.frame = g.frame;
    cp.inv_w = 1.0 / g.w;
    cp.w = g.w;
    for (int j = 0; j < g.d; ++j) {
        cp.gmin[j] = g.gmin[j];
        cp.ng[j] = g.ng[j];
        cp.stride[j] = g.stride[j];
    }
    return cp;
}

// Cell coordinate in dimension j of a point whose offset from the grid's
// lower corner is a = fl64(x_j - g_min_j): c_j = floor(q) for q = fl64(a *
// (1 / w)), clamped to [0, |g_j| - 1].  The floor is taken on q's bits
// with integer instructions (the FP64 pipe is the bottleneck of the cell
// pass): q < 1, including -0 and every negative q, gives 0; q >= 2^31
// exceeds |g_j| - 1 < 2^31; otherwise, with q = m 2^(e - 52) for the 53-bit
// significand m and exponent e in [0, 30], floor(q) = m >> (52 - e).
__device__ __forceinline__ int64_t cell_of_offset(double a, int j, const CellParams &cp) {
    const double q = __dmul_rn(a, cp.inv_w);
    const uint64_t b = (uint64_t)__double_as_longlong(q);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    int64_t c;
    if ((b >> 63) != 0 || e < 0)
        c = 0;
    else if (e > 30)
        c = cp.ng[j] - 1;
    else
        c = (int64_t)(((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> (52 - e));
    return c > cp.ng[j] - 1 ? cp.ng[j] - 1 : c;
}

// Cell coordinate of point p in dimension j: c_j = floor((x_j - g_min_j) *
// (1 / w)) in FP64, clamped to the grid.  Every part of the index computes
// a point's cell with this one formula (cell_of_offset).
__device__ __forceinline__ int64_t cell_coord(const double *p, int j, const CellParams &cp) {
    return cell_of_offset(__dsub_rn(p[j], cp.gmin[j]), j, cp);
}

// FP32 record coordinate of offset a = fl64(x_j - g_min_j) in cell
// coordinate c: grid frame y = fl32(a); cell frame y = fl32(a - fl64(4 K w))
// with K = floor(c / 4).
__device__ __forceinline__ float rec_coord(double a, int64_t c, const CellParams &cp) {
    double y = a;
    if (cp.frame == SJ_FRAME_CELL) y = __dsub_rn(a, __dmul_rn((double)(4 * (c >> 2)), cp.w));
    return __double2float_rn(y);
}

// Linear cell id of point p: id = sum_j c_j * stride_j (dimension 1 fastest).
__device__ __forceinline__ uint64_t linear_cell(const double *p, const CellParams &cp) {
    uint64_t id = 0;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j)
        if (j < cp.d) id += (uint64_t)cell_coord(p, j, cp) * cp.stride[j];
    return id;
}

// Accumulates per-dimension min / max (order keys) of points i0, i0 + step,
// ... below n into minmax[2j], minmax[2j + 1] and sets bit 0 of *flag when a
// coordinate is NaN or infinite.  Called by every thread of full warps.
template <int MAXD = kMaxDim>
__device__ __forceinline__ void bounds_accumulate(const double *__restrict__ pts, uint64_t n, int d,
                                                  uint64_t i0, uint64_t step,
                                                  unsigned long long *minmax, uint32_t *flag) {
    unsigned long long lo[MAXD], hi[MAXD];
#pragma unroll
    for (int j = 0; j < MAXD; ++j) { lo[j] = ~0ULL; hi[j] = 0ULL; }
    bool bad = false;
    for (uint64_t i = i0; i < n; i += step) {
#pragma unroll
        for (int j = 0; j < MAXD; ++j) {
            if (j < d) {
                const double x = pts[i * d + j];
                const unsigned long long b = (unsigned long long)__double_as_longlong(x);
                bad |= (b & 0x7ff0000000000000ULL) == 0x7ff0000000000000ULL;
                const unsigned long long k = order_key(x);
                lo[j] = k < lo[j] ? k : lo[j];
                hi[j] = k > hi[j] ? k : hi[j];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAXD; ++j) {
        if (j < d) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[j], o);
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[j], o);
                lo[j] = a < lo[j] ? a : lo[j];
                hi[j] = b > hi[j] ? b : hi[j];
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&minmax[2 * j], lo[j]);
                atomicMax(&minmax[2 * j + 1], hi[j]);
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Shared-memory words for the occupancy bitmaps in cells_block: when all d
// bitmaps fit (d * mwords words), bits collect per block and are merged
// into M with one atomicOr per non-zero word and block.
constexpr uint32_t kCellsSmemWords = 2048;

// Coordinates of the cell with linear id `id` (id = sum_j c_j stride_j with
// 0 <= c_j < |g_j|, dimension 1 fastest): the mixed-radix digits of id,
// equal to the coordinates linear_cell combined.
__device__ __forceinline__ void coords_of_id(uint64_t id, const CellParams &cp, int64_t *c) {
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
        if (j < cp.d) {
            const uint64_t g = (uint64_t)cp.ng[j];
            if ((id >> 32) == 0) {
                const uint32_t r = (uint32_t)id, q = r / (uint32_t)g;
                c[j] = (int64_t)(r - q * (uint32_t)g);
                id = q;
            } else {
                const uint64_t q = id / g;
                c[j] = (int64_t)(id - q * g);
                id = q;
            }
        }
    }
}

// Cell coordinates of the non-empty cells h = h0, h0 + step, ... below nc
// into cc (d per cell), and their bits in the occupancy bitmaps M_j (word
// j * mwords + c_j / 32).  The coordinates are the digits of the cell's
// linear id B[h] (FROM_KEY) or, for cells ordered by coordinate tuple (no
// B), recomputed from one of the cell's points with the formula of
// linear_cell.  sm: shared memory of kCellsSmemWords words; the bits
// collect there when the d bitmaps fit.  A word is read before its
// atomicOr, so that a bit already set costs no atomic (a stale read only
// costs a redundant one).  Every thread of the block calls this (it has
// barriers).
template <bool FROM_KEY>
__device__ __forceinline__ void cells_block(const double *__restrict__ pts,
                                            const uint32_t *__restrict__ A,
                                            const uint32_t *__restrict__ G,
                                            const uint64_t *__restrict__ B, uint64_t nc,
                                            uint64_t h0, uint64_t step, const CellParams &cp,
                                            uint32_t mwords, int32_t *__restrict__ cc,
                                            uint32_t *__restrict__ M, uint32_t *sm) {
    const uint64_t mw = (uint64_t)cp.d * mwords;
    const bool local = mw <= kCellsSmemWords;
    if (local) {
        for (uint32_t k = threadIdx.x; k < mw; k += blockDim.x) sm[k] = 0u;
        __syncthreads();
    }
    uint32_t *bits = local ? sm : M;
    for (uint64_t h = h0; h < nc; h += step) {
        int64_t c[kMaxDim];
        if (FROM_KEY) {
            coords_of_id(B[h], cp, c);
        } else {
            const double *p = pts + (uint64_t)A[G[h]] * cp.d;
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j)
                if (j < cp.d) c[j] = cell_coord(p, j, cp);
        }
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) {
            if (j < cp.d) {
                cc[h * cp.d + j] = (int32_t)c[j];
                uint32_t *w = &bits[(uint64_t)j * mwords + (uint64_t)(c[j] >> 5)];
                const uint32_t bit = 1u << (c[j] & 31);
                const uint32_t seen = local ? *w : __ldcg(w);
                if ((seen & bit) == 0) atomicOr(w, bit);
            }
        }
    }
    if (local) {
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < mw; k += blockDim.x)
            if (sm[k]) atomicOr(&M[k], sm[k]);
    }
}

// FP32 record of the point at cell-order position k, then the point id and
// zero padding up to rs floats.  Grid frame: y_j = fl32(x_j - g_min_j).
// Cell frame: y_j = fl32(fl64(x_j - g_min_j) - fl64(4 K_j w)) with
// K_j = floor(c_j / 4) for the point's cell coordinate c_j (the formula of
// linear_cell), so that y_j lies within about four cell sides of 0 at any
// extent of the grid.
__device__ __forceinline__ void write_rec32(const double *__restrict__ pts,
                                            const uint32_t *__restrict__ A, uint64_t k,
                                            const CellParams &cp, int rs, float *__restrict__ rec) {
    const uint32_t i = A[k];
    const double *p = pts + (uint64_t)i * cp.d;
    float *r = rec + k * rs;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
        if (j < cp.d) {
            const double a = __dsub_rn(p[j], cp.gmin[j]);
            r[j] = rec_coord(a, cp.frame == SJ_FRAME_CELL ? cell_of_offset(a, j, cp) : 0, cp);
        }
    }
    r[cp.d] = __uint_as_float(i);
    for (int j = cp.d + 1; j < rs; ++j) r[j] = 0.0f;
}

// FP64 record: x_0 .. x_{d-1}, the point id, zero padding up to rs doubles.
__device__ __forceinline__ void write_rec64(const double *__restrict__ pts,
                                            const uint32_t *__restrict__ A, uint64_t k, int d,
                                            int rs, double *__restrict__ rec) {
    const uint32_t i = A[k];
    const double *p = pts + (uint64_t)i * d;
    double *r = rec + k * rs;
    for (int j = 0; j < d; ++j) r[j] = p[j];
    r[d] = __longlong_as_double((long long)i);
    for (int j = d + 1; j < rs; ++j) r[j] = 0.0;
}

}  // namespace sj
