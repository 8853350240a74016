// join_dev.cuh -- device helpers shared by the search-and-refine kernels:
// the main kernel (join.cu) and the one for more than 8 dimensions
// (hd_join.cu): packed FP32 pair arithmetic, the row templates of the
// adjacent-cell search (Section IV-D) under UNICOMP (Section V-B), and the
// lookup of a row's candidate range.
#pragma once

#include "sj_internal.cuh"

namespace sj {

namespace {

// Packed FP32 pair arithmetic (sm_100+ f32x2 instructions), round to nearest.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Row templates of the search, precomputed on the host per (d, UNICOMP)
// and read with one load per template.  Entry t describes template t
// relative to the query cell c:
//   bits 0-1  x range: 0 the home cell only, 1 x - 1 only, 2 x + 1 only,
//             3 x - 1 .. x + 1;
//   bits 2-5  gate: the template is active when bit `gate` of the cell's
//             odd-coordinate mask is set (gate < 8), always (gate = 8);
//   bits 6-19 offset + 1 of dimensions 2..d (2 bits each).
//   UNICOMP: t = 0 home cell; t = 1, 2 stage 0 (x - 1, x + 1); then, for
//   stage k = 1..d-1, 2 * 3^(k-1) rows with dimension k at c_k -+ 1,
//   dimensions 1..k-1 anywhere in c -+ 1, dimensions above k equal to c.
//   Stage k is active when c_k is odd (Section V-B, generalised to n
//   dimensions).  Full search: t in [0, 3^(d-1)) enumerates all rows.
template <int D, bool UNI>
__device__ __forceinline__ bool row_of(int t, const int32_t *c, uint32_t odd, uint32_t occ, const JoinArgs &a,
                                       int32_t &xlo, int32_t &xhi, int32_t *b) {
    const uint32_t e = __ldg(&a.tmpl[t]);
    const uint32_t gate = (e >> 2) & 15u;
    if (gate < 8 && !((odd >> gate) & 1u)) return false;
    const uint32_t xm = e & 3u;
    xlo = c[0] + (xm == 2 ? 1 : (xm == 0 ? 0 : -1));
    xhi = c[0] + (xm == 1 ? -1 : (xm == 0 ? 0 : 1));
#pragma unroll
    for (int j = 1; j < D; ++j) b[j] = c[j] + (int32_t)((e >> (6 + 2 * (j - 1))) & 3u) - 1;
    if (xlo < 0) xlo = 0;
    if (xhi > a.ng[0] - 1) xhi = a.ng[0] - 1;
    if (xlo > xhi) return false;
#pragma unroll
    for (int j = 1; j < D; ++j)
        if (!((occ >> (3 * (j - 1) + ((e >> (6 + 2 * (j - 1))) & 3u))) & 1u)) return false;
    return true;
}

// First position in B[0, n) whose value is >= key.
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *__restrict__ B, uint32_t n,
                                                    uint64_t key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&B[mid]) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// First cell in [0, n) whose coordinate tuple is not below (b_{D-1}, ...,
// b_1, x), compared from dimension D down to dimension 1: the order of the
// linear ids, for grids whose linear ids do not fit in 64 bits.
template <int D>
__device__ __forceinline__ uint32_t lower_bound_tuple(const int32_t *__restrict__ cc, uint32_t n,
                                                      const int32_t *b, int32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const int32_t *t = cc + (uint64_t)mid * D;
        int cmp = 0;
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            const int32_t tj = __ldg(&t[j]);
            const int32_t kj = j ? b[j] : x;
            if (cmp == 0) cmp = tj < kj ? -1 : (tj > kj ? 1 : 0);
        }
        if (cmp < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Candidate ranges of a query cell with coordinates c (odd: their parity
// bits): one entry per row template that survives the M_j clip and holds
// points, written to rt as (first record, running candidate count); K is
// the number of candidates.
// Under UNICOMP the table holds the home row (template 0), the two stage-0
// cells (1, 2; gate 0) and, per stage k = 1 .. D-1, 2 * 3^(k-1) rows from
// template 3^(k-1) + 2 on (gate k).  Only the stages whose gate coordinate
// is odd take part, so the lanes are mapped onto those templates alone:
// at 6-D about 123 of 245, half the passes.
template <int D>
__device__ __forceinline__ int active_template(uint32_t odd, uint32_t r) {
    if (r == 0) return 0;
    --r;
    if (odd & 1u) {
        if (r < 2) return 1 + (int)r;
        r -= 2;
    }
    uint32_t p = 1;   // 3^(k-1)
#pragma unroll
    for (int k = 1; k < D; ++k) {
        if ((odd >> k) & 1u) {
            if (r < 2 * p) return (int)(p + 2 + r);
            r -= 2 * p;
        }
        p *= 3;
    }
    return -1;
}

template <int D>
__device__ __forceinline__ uint32_t active_templates(uint32_t odd) {
    uint32_t n = 1 + ((odd & 1u) ? 2u : 0u), p = 1;
#pragma unroll
    for (int k = 1; k < D; ++k) {
        if ((odd >> k) & 1u) n += 2 * p;
        p *= 3;
    }
    return n;
}

template <int D, bool UNI>
__device__ __forceinline__ void build_ranges(const int32_t *c, uint32_t odd, const JoinArgs &a,
                                             uint32_t n_cells, int lane, uint2 *rt,
                                             uint32_t &nranges, uint32_t &K) {
    nranges = 0;
    K = 0;
    // slab occupancy c_j - 1, c_j, c_j + 1 of dimensions 2..D (in the grid
    // and marked in M_j): bit 3 (j - 1) + offset + 1, one lane per bit
    uint32_t occ;
    {
        bool ok = false;
        if (lane < 3 * (D - 1)) {
            const int j = 1 + lane / 3;
            int32_t cj = 0;
#pragma unroll
            for (int jj = 1; jj < D; ++jj) if (jj == j) cj = c[jj];
            const int32_t bj = cj + lane % 3 - 1;
            if (bj >= 0 && bj < a.ng[j]) {
                const uint32_t w = __ldg(&a.M[(uint64_t)j * a.mwords + ((uint32_t)bj >> 5)]);
                ok = (w >> (bj & 31)) & 1u;
            }
        }
        occ = __ballot_sync(0xffffffffu, ok);
    }
    const int n_t = UNI ? (int)active_templates<D>(odd) : a.n_templates;
    for (int t0 = 0; t0 < n_t; t0 += 32) {
        const int t = UNI ? (t0 + lane < n_t ? active_template<D>(odd, (uint32_t)(t0 + lane)) : -1)
                          : (t0 + lane < n_t ? t0 + lane : -1);
        uint32_t beg = 0, len = 0;
        int32_t xlo, xhi, b[D];
        if (t >= 0 && row_of<D, UNI>(t, c, odd, occ, a, xlo, xhi, b)) {
            uint64_t base = 0;
#pragma unroll
            for (int j = 1; j < D; ++j) base += (uint64_t)b[j] * a.stride[j];
            const uint64_t id_lo = base + (uint64_t)xlo, id_hi = base + (uint64_t)xhi;
            uint32_t e;
            if (a.dense) {
                beg = __ldg(&a.lut[id_lo]);
                e = __ldg(&a.lut[id_hi + 1]);
            } else if (a.tuple) {
                const uint32_t hl = lower_bound_tuple<D>(a.cc, n_cells, b, xlo);
                const uint32_t hh = lower_bound_tuple<D>(a.cc, n_cells, b, xhi + 1);
                beg = __ldg(&a.G[hl]);
                e = __ldg(&a.G[hh]);
            } else {
                const uint32_t hl = lower_bound_u64(a.B, n_cells, id_lo);
                const uint32_t hh = lower_bound_u64(a.B, n_cells, id_hi + 1);
                beg = __ldg(&a.G[hl]);
                e = __ldg(&a.G[hh]);
            }
            len = e - beg;
        }
        const unsigned nz = __ballot_sync(0xffffffffu, len > 0);
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (len > 0) rt[nranges + __popc(nz & ((1u << lane) - 1u))] = make_uint2(beg, K + incl);
        nranges += __popc(nz);
        K += __shfl_sync(0xffffffffu, incl, 31);
    }
}

}  // namespace

}  // namespace sj
