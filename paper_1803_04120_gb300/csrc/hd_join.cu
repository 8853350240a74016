// hd_join.cu -- the search-and-refine kernel for points of more than 8
// dimensions (up to 16).  The grid covers the six dimensions with the most
// cells (index.cu, build_index_hd); the search refines on every coordinate.
#include "join_dev.cuh"

namespace sj {

namespace {

// The exact predicate for the high-dimensional kernel's rechecks: a
// function of its own, so that the main kernels' non-inlined recheck keeps
// its register budget.
__device__ __noinline__ bool exact_member_hd(const double *__restrict__ a,
                                             const double *__restrict__ b, int d, double E2) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        const double t = __dsub_rn(a[j], b[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s <= E2;
}

// High-dimensional search (points of more than kMaxDim dimensions): the
// grid covers kHdGridDims of them.  A warp takes one work item at a time,
// builds its candidate ranges like the main kernel, stages the item's
// queries (records of all dfull coordinates) in shared memory, and lets each
// lane take every 32nd candidate of each range, read straight from the
// cell-ordered records in global memory, and compare it with every query.
// FP32: the expanded-form sum (EXP: |z_q|^2 + |z_p|^2 - 2 z_p . z_q about
// an origin at the home cell centre in the grid dimensions and at the
// middle of the data range in the others, one fma per coordinate) or the
// difference form (two per coordinate, where the expanded form has no
// usable margin), against [lo32, hi32] (margin.cu); values in between are
// rechecked with the exact FP64 predicate on the input points, in a
// warp-uniform branch.  FP64: the exact predicate on the FP64 records.
// Hits are written after one atomic reservation per query and 32
// candidates.  There are no waits, so no time limits.
template <bool F32, bool UNI, int G4, bool EXP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2)
    hd_join_kernel(const JoinArgs a, const uint32_t *counts) {
    // DW = 4 G4 >= d coordinates take part; those past d are zero on both
    // sides, and an exact zero term leaves every sum (FP32 or FP64) unchanged
    constexpr int K = kHdGridDims;
    constexpr int DW = 4 * G4;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * a.sm_warp;
    uint2 *rt = reinterpret_cast<uint2 *>(wbase);
    // staged queries (FP32): the DW floats y (difference form) or m = -2 z
    // (expanded form) then |z|^2 and three pads, read 16 bytes per four
    // coordinates and paired in registers (the shared-memory pipe is what
    // limits these loops); FP64: the DW doubles
    unsigned char *qs = wbase + a.sm_ranges;
    float *origin = reinterpret_cast<float *>(wbase + a.sm_ranges + a.sm_queries);
    constexpr int QF = DW + 4;   // floats per staged expanded-form query
    const int dd = a.dfull, rs = a.rsd;
    const uint32_t n_cells = *a.ccells;
    uint32_t item_end = a.item_end;
    if (counts[1] < item_end) item_end = counts[1];
    const unsigned lt = (1u << lane) - 1u;
    constexpr unsigned long long kMult = UNI ? 2ull : 1ull;
    unsigned long long evals = 0, rechecks = 0;

    // one classified hit per lane: reservation by ballot, then the writes
    auto emit = [&](bool hit, uint32_t qid, uint32_t cid) {
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (!m) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.counter[0], (unsigned long long)__popc(m) * kMult);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (hit && !a.count_only) {
            const unsigned long long at = base + (unsigned long long)__popc(m & lt) * kMult;
            if (at < a.cap) a.out[at] = make_uint2(qid, cid);
            if (UNI && at + 1 < a.cap) a.out[at + 1] = make_uint2(cid, qid);
        }
    };

    for (;;) {
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(a.work, 1u);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        const uint64_t item = (uint64_t)a.item_begin + (uint64_t)pos * a.item_stride;
        if (item >= item_end) break;
        const uint2 it = a.items[item];
        const uint32_t h = it.x;
        const uint32_t cbeg = __ldg(&a.qG[h]), cend = __ldg(&a.qG[h + 1]);
        const uint32_t home_len = cend - cbeg;
        const uint32_t ql0 = it.y * kQueryBlock;
        const uint32_t q0 = cbeg + ql0;
        const uint32_t nq = min((uint32_t)kQueryBlock, cend - q0);
        int32_t c[K];
        uint32_t odd = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            c[j] = __ldg(&a.qcc[(uint64_t)h * K + j]);
            odd |= ((uint32_t)c[j] & 1u) << j;
        }
        __syncwarp();   // the previous item's ranges and queries are no longer read
        uint32_t nranges, kc;
        build_ranges<K, UNI>(c, odd, a, n_cells, lane, rt, nranges, kc);
        uint32_t qid_l = 0;
        if (EXP) {
            // the origin: home cell centre in a grid dimension (as in the
            // grid frame), the middle of the data range in the others
            if (lane < DW) {
                const int t = lane < dd ? (int)((a.hgrid4 >> (4 * lane)) & 0xfull) : 15;
                int32_t ct = 0;
#pragma unroll
                for (int tt = 0; tt < K; ++tt) if (tt == t) ct = c[tt];
                origin[lane] = t < K ? ((float)ct + 0.5f) * a.w32 : (lane < dd ? __ldg(&a.hmid[lane]) : 0.0f);
            }
            __syncwarp();
        }
        if (lane < (int)nq) {
            if (F32 && EXP) {
                const float *r = a.recd32 + (size_t)(q0 + lane) * rs;
                float *qd = reinterpret_cast<float *>(qs) + (size_t)lane * QF;
                float pp = 0.0f;
#pragma unroll
                for (int j = 0; j < DW; ++j) {
                    const float z = j < dd ? __fsub_rn(r[j], origin[j]) : 0.0f;
                    pp = __fmaf_rn(z, z, pp);
                    qd[j] = -2.0f * z;
                }
                qd[DW] = pp;
                qd[DW + 1] = qd[DW + 2] = qd[DW + 3] = 0.0f;
                qid_l = __float_as_uint(r[dd]);
            } else if (F32) {
                const float *r = a.recd32 + (size_t)(q0 + lane) * rs;
                float *qd = reinterpret_cast<float *>(qs) + (size_t)lane * QF;
#pragma unroll
                for (int j = 0; j < DW; ++j) qd[j] = j < dd ? r[j] : 0.0f;
                qid_l = __float_as_uint(r[dd]);
            } else {
                const double *r = a.recd64 + (size_t)(q0 + lane) * rs;
                double *qd = reinterpret_cast<double *>(qs) + (size_t)lane * DW;
#pragma unroll
                for (int j = 0; j < DW; ++j) qd[j] = j < dd ? r[j] : 0.0;
                qid_l = (uint32_t)__double_as_longlong(r[dd]);
            }
        }
        __syncwarp();
        if (lane == 0)
            evals += UNI ? (uint64_t)nq * (kc - home_len) + (uint64_t)nq * (home_len - 1) -
                               (uint64_t)nq * ql0 - (uint64_t)nq * (nq - 1) / 2
                         : (uint64_t)nq * kc;
        if (UNI) {
            // the self-pair of every query, once
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&a.counter[0], (unsigned long long)nq);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (!a.count_only && lane < (int)nq && base + lane < a.cap)
                a.out[base + lane] = make_uint2(qid_l, qid_l);
        }
        uint32_t kstart = 0;
        for (uint32_t ri = 0; ri < nranges; ++ri) {
            const uint2 rg = rt[ri];
            const uint32_t len = rg.y - kstart;
            if (F32) {
                // two candidates per lane (p and p + 32), packed as f32x2;
                // a slot past the range holds coordinates far outside the
                // data (its sum overflows to +inf, or is NaN: never at or
                // below hi32), so the comparison needs no per-query
                // validity test
                for (uint32_t p0 = 0; p0 < len; p0 += 64) {
                    uint32_t cid[2] = {0xffffffffu, 0xffffffffu}, kp[2];
                    float4 y4[2][G4];
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const uint32_t p = p0 + 32 * h2 + lane;
                        kp[h2] = kstart + p;
                        const float far = p < len ? 0.0f : 1.0e30f;
#pragma unroll
                        for (int g = 0; g < G4; ++g) y4[h2][g] = make_float4(far, far, far, far);
                        if (p < len) {
                            const float *r = a.recd32 + (size_t)(rg.x + p) * rs;
#pragma unroll
                            for (int g = 0; g < G4; ++g) y4[h2][g] = *reinterpret_cast<const float4 *>(r + 4 * g);
                            cid[h2] = __float_as_uint(r[dd]);
                        }
                    }
                    f2_t yy[DW];
#pragma unroll
                    for (int g = 0; g < G4; ++g) {
                        const float4 u = y4[0][g], v = y4[1][g];
                        const int j = 4 * g;
                        yy[j] = f2_pack(j < dd ? u.x : 0.f, j < dd ? v.x : 0.f);
                        yy[j + 1] = f2_pack(j + 1 < dd ? u.y : 0.f, j + 1 < dd ? v.y : 0.f);
                        yy[j + 2] = f2_pack(j + 2 < dd ? u.z : 0.f, j + 2 < dd ? v.z : 0.f);
                        yy[j + 3] = f2_pack(j + 3 < dd ? u.w : 0.f, j + 3 < dd ? v.w : 0.f);
                    }
                    f2_t qq = f2_pack(0.0f, 0.0f);
                    if (EXP) {
                        // z = fl(y - o) (exact negation, one rounding) and
                        // |z|^2 of both candidates
#pragma unroll
                        for (int j = 0; j < DW; ++j) {
                            const float no = -origin[j];
                            yy[j] = f2_add(yy[j], f2_pack(no, no));
                            qq = f2_fma(yy[j], yy[j], qq);
                        }
                    }
                    // the UNICOMP home-cell rule, the band rechecks and the
                    // writes of one query, in the rare branch where a lane
                    // has a hit
                    auto handle = [&](uint32_t qi, const float *sv) {
                        const uint32_t qid = __shfl_sync(0xffffffffu, qid_l, qi);
                        bool hit[2], band[2];
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const bool cand = !UNI || kp[h2] >= home_len || kp[h2] > ql0 + qi;
                            hit[h2] = cand && sv[h2] <= a.hi32;
                            band[h2] = hit[h2] && !(sv[h2] <= a.lo32);
                        }
                        if (__any_sync(0xffffffffu, band[0] || band[1])) {
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                if (band[h2]) {
                                    hit[h2] = exact_member_hd(a.ptsd + (size_t)qid * dd,
                                                              a.ptsd + (size_t)cid[h2] * dd, dd, a.E2);
                                    ++rechecks;
                                }
                            }
                        }
                        emit(hit[0], qid, cid[0]);
                        emit(hit[1], qid, cid[1]);
                    };
                    // s32 of query q against this lane's two candidates
                    auto sum_of = [&](uint32_t q, float *sv) {
                        const float4 *qd =
                            reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(qs) + (size_t)q * QF);
                        f2_t acc0 = f2_pack(0.0f, 0.0f), acc1 = acc0;
                        if (EXP) {
                            // fl(qq + pp), then the m_j z_j terms in two
                            // chains (even and odd j) added at the end
                            const float pp = qd[G4].x;
                            acc0 = f2_add(qq, f2_pack(pp, pp));
#pragma unroll
                            for (int g = 0; g < G4; ++g) {
                                const float4 m4 = qd[g];   // m_4g .. m_4g+3, paired in registers
                                acc0 = f2_fma(f2_pack(m4.x, m4.x), yy[4 * g], acc0);
                                acc1 = f2_fma(f2_pack(m4.y, m4.y), yy[4 * g + 1], acc1);
                                acc0 = f2_fma(f2_pack(m4.z, m4.z), yy[4 * g + 2], acc0);
                                acc1 = f2_fma(f2_pack(m4.w, m4.w), yy[4 * g + 3], acc1);
                            }
                        } else {
                            // fl(q - y)^2 in two running fma sums, even and
                            // odd coordinates, added at the end (the margin
                            // holds for any grouping, margin.cu); the
                            // difference as fma(y, -1, q) rounds once like q - y
                            const f2_t neg1 = f2_pack(-1.0f, -1.0f);
#pragma unroll
                            for (int g = 0; g < G4; ++g) {
                                const float4 q4 = qd[g];   // q_4g .. q_4g+3, paired in registers
                                const f2_t t0 = f2_fma(yy[4 * g], neg1, f2_pack(q4.x, q4.x));
                                acc0 = f2_fma(t0, t0, acc0);
                                const f2_t t1 = f2_fma(yy[4 * g + 1], neg1, f2_pack(q4.y, q4.y));
                                acc1 = f2_fma(t1, t1, acc1);
                                const f2_t t2 = f2_fma(yy[4 * g + 2], neg1, f2_pack(q4.z, q4.z));
                                acc0 = f2_fma(t2, t2, acc0);
                                const f2_t t3 = f2_fma(yy[4 * g + 3], neg1, f2_pack(q4.w, q4.w));
                                acc1 = f2_fma(t3, t3, acc1);
                            }
                        }
                        f2_unpack(f2_add(acc0, acc1), sv[0], sv[1]);
                    };
                    // two queries per vote: hits are a few in 1e4
                    // comparisons, and the vote and its branch per query
                    // were the loop's largest stall after the arithmetic
                    for (uint32_t qi = 0; qi < nq; qi += 2) {
                        const uint32_t qb = qi + 1 < nq ? qi + 1 : qi;
                        float sa[2], sb[2];
                        sum_of(qi, sa);
                        sum_of(qb, sb);
                        const bool ha = sa[0] <= a.hi32 || sa[1] <= a.hi32;
                        const bool hb = qb != qi && (sb[0] <= a.hi32 || sb[1] <= a.hi32);
                        if (!__any_sync(0xffffffffu, ha || hb)) continue;
                        if (__any_sync(0xffffffffu, ha)) handle(qi, sa);
                        if (__any_sync(0xffffffffu, hb)) handle(qb, sb);
                    }
                }
            } else {
                for (uint32_t p0 = 0; p0 < len; p0 += 32) {
                    const uint32_t p = p0 + lane;
                    const bool valid = p < len;
                    const uint32_t kpos = kstart + p;   // position in the item's candidate list
                    double y[DW];
                    uint32_t cid = 0xffffffffu;
#pragma unroll
                    for (int j = 0; j < DW; ++j) y[j] = 0.0;
                    if (valid) {
                        const double *r = a.recd64 + (size_t)(rg.x + p) * rs;
#pragma unroll
                        for (int j = 0; j < DW; ++j)
                            if (j < dd) y[j] = r[j];
                        cid = (uint32_t)__double_as_longlong(r[dd]);
                    }
                    for (uint32_t qi = 0; qi < nq; ++qi) {
                        const uint32_t qid = __shfl_sync(0xffffffffu, qid_l, qi);
                        const bool cand = valid && (!UNI || kpos >= home_len || kpos > ql0 + qi);
                        const double *qd = reinterpret_cast<const double *>(qs) + (size_t)qi * DW;
                        // the exact predicate, in dimension order (zero terms add nothing)
                        double sum = 0.0;
#pragma unroll
                        for (int j = 0; j < DW; ++j) {
                            const double t = __dsub_rn(qd[j], y[j]);
                            sum = __dadd_rn(sum, __dmul_rn(t, t));
                        }
                        emit(cand && sum <= a.E2, qid, cid);
                    }
                }
            }
            kstart = rg.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
    if (lane == 0) {
        if (evals) atomicAdd(&a.counter[1], evals);
        if (rechecks) atomicAdd(&a.counter[2], rechecks);
    }
}

// The high-dimensional kernel evaluates 12 (d <= 12) or 16 coordinates.
template <int G4>
JoinKernelFn pick_hd(bool f32, bool uni, bool exp) {
    if (f32 && exp) return uni ? hd_join_kernel<true, true, G4, true> : hd_join_kernel<true, false, G4, true>;
    if (f32) return uni ? hd_join_kernel<true, true, G4, false> : hd_join_kernel<true, false, G4, false>;
    return uni ? hd_join_kernel<false, true, G4, false> : hd_join_kernel<false, false, G4, false>;
}

}  // namespace

JoinKernelFn hd_kernel_fn(int d, bool f32, bool uni, bool exp) {
    if (d <= 12) return pick_hd<3>(f32, uni, exp);
    if (d <= kMaxPointDim) return pick_hd<4>(f32, uni, exp);
    return nullptr;
}

}  // namespace sj
