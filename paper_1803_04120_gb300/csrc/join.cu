// join.cu -- persistent search-and-refine kernel (Section IV-D, IV-E, V-B).
//
// Work decomposition.  A work item is (non-empty cell h, block of up to 32
// of its points); items are taken from a global cursor by whole warps, so
// heavy cells are spread over many warps.  For its item a warp:
//   1. builds the candidate ranges: the adjacent cells the query cell must
//      search (Section IV-D), chosen by UNICOMP (Section V-B) or all 3^n of
//      them (Algorithm 1).  Cells adjacent along dimension 1 have consecutive
//      linear ids, so a "row" of up to three cells that agree in dimensions
//      2..n is one contiguous range of the cell-ordered records; a row is
//      skipped when M_j marks one of its fixed coordinates as empty, and is
//      looked up with two loads of the dense table or two binary searches of
//      B.  The home cell is range 0.
//   2. streams the candidates through shared memory in chunks of 64: every
//      range piece of a chunk is one cp.async.bulk copy (16-byte aligned
//      records) completing on a per-warp mbarrier, double buffered so the
//      next chunk is in flight while the current one is compared.
//   3. compares: lanes own candidates (two each), the item's query points
//      are broadcast from shared memory.  FP32 mode computes the squared
//      distance with packed f32x2 arithmetic and classifies it against the
//      proven margin [lo32, hi32]; only values inside it are recomputed with
//      the exact FP64 predicate.  FP64 mode evaluates the predicate directly.
//   4. emits: under UNICOMP each hit (p, q) gives (p, q) and (q, p); in the
//      home cell only q >= p is compared and the self-pair is emitted once.
//      Pairs are staged per warp in shared memory (ballot-free warp scan for
//      the offsets) and written out in coalesced blocks after one atomic
//      reservation per flush.
// Waits on mbarriers are bounded by a time limit; on expiry the warp records
// an error bit, waits (bounded) for its copies in flight and leaves.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kCPL = 2;                    // candidates per lane
constexpr int kChunk = 32 * kCPL;          // candidates per chunk
constexpr int kEmit = 512;                 // staged pairs per warp

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of an mbarrier: false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

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
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The exact predicate of Section III in FP64: every operation rounded to
// nearest on its own, no contraction.
template <int D>
__device__ __forceinline__ bool exact_member(const double *__restrict__ a,
                                             const double *__restrict__ b, double E2) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        double t = __dsub_rn(a[j], b[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s <= E2;
}

// Powers of three for decoding row templates.
__constant__ uint32_t c_pow3[kMaxDim + 1] = {1, 3, 9, 27, 81, 243, 729, 2187, 6561};

// Row template t of the search, for a query cell with coordinates c:
// outputs the x range [xlo, xhi] and the offsets of dimensions 1..D-1, or
// false when the template is inactive or leaves the grid.
//   UNICOMP: t = 0 home cell; t = 1, 2 stage 0 (x - 1, x + 1); then, for
//   stage k = 1..D-1, 2 * 3^(k-1) rows with dimension k at c_k -+ 1,
//   dimensions 1..k-1 anywhere in c -+ 1, dimensions above k equal to c.
//   Stage k is active when c_k is odd (Section V-B, generalised to n
//   dimensions).  Full search: t in [0, 3^(D-1)) enumerates all rows.
template <int D, bool UNI>
__device__ __forceinline__ bool row_of(int t, const int32_t *c, uint32_t odd, const JoinArgs &a,
                                       int32_t &xlo, int32_t &xhi, int32_t *b) {
#pragma unroll
    for (int j = 1; j < D; ++j) b[j] = c[j];
    xlo = c[0] - 1;
    xhi = c[0] + 1;
    if (UNI) {
        if (t == 0) {
            xlo = xhi = c[0];
        } else if (t <= 2) {
            if (!(odd & 1u)) return false;
            xlo = xhi = (t == 1) ? c[0] - 1 : c[0] + 1;
        } else {
            uint32_t u = (uint32_t)t - 3;
            int k = 1;
#pragma unroll
            for (int kk = 1; kk < D; ++kk)
                if (u >= c_pow3[kk] - 1) k = kk + 1;
            if (k >= D) return false;
            if (!((odd >> k) & 1u)) return false;
            uint32_t v = u - (c_pow3[k - 1] - 1);
            uint32_t p = c_pow3[k - 1];
            b[k] = c[k] + ((v / p) ? 1 : -1);
            uint32_t rem = v % p;
#pragma unroll
            for (int j = 1; j < D; ++j) {
                if (j < k) {
                    b[j] = c[j] + (int32_t)(rem % 3) - 1;
                    rem /= 3;
                }
            }
        }
    } else {
        uint32_t rem = (uint32_t)t;
#pragma unroll
        for (int j = 1; j < D; ++j) {
            b[j] = c[j] + (int32_t)(rem % 3) - 1;
            rem /= 3;
        }
    }
    if (xlo < 0) xlo = 0;
    if (xhi > a.ng[0] - 1) xhi = a.ng[0] - 1;
    if (xlo > xhi) return false;
#pragma unroll
    for (int j = 1; j < D; ++j) {
        if (b[j] < 0 || b[j] >= a.ng[j]) return false;
        uint32_t w = a.M[(uint64_t)j * a.mwords + ((uint32_t)b[j] >> 5)];
        if (!((w >> (b[j] & 31)) & 1u)) return false;   // M_j: no point in that slab
    }
    return true;
}

// First position in B[0, n) whose value is >= key.
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *__restrict__ B, uint32_t n,
                                                    uint64_t key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&B[mid]) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Per-warp shared-memory carve-up.
struct WarpSmem {
    uint2 *ranges;        // (begin in cell order, flat end)
    unsigned char *q;     // query records
    unsigned char *buf[2];
    uint2 *emit;
    uint64_t *bar;        // two mbarriers
};

__device__ __forceinline__ WarpSmem carve(unsigned char *base, const JoinArgs &a, int warp) {
    WarpSmem w;
    unsigned char *p = base + (size_t)warp * a.sm_warp;
    w.bar = reinterpret_cast<uint64_t *>(p);
    p += 16;
    w.ranges = reinterpret_cast<uint2 *>(p);
    p += a.sm_ranges;
    w.q = p;
    p += a.sm_queries;
    w.buf[0] = p;
    p += a.sm_chunk;
    w.buf[1] = p;
    p += a.sm_chunk;
    w.emit = reinterpret_cast<uint2 *>(p);
    return w;
}

struct Emitter {
    uint32_t fill = 0;
};

__device__ __forceinline__ void flush(Emitter &em, const WarpSmem &ws, const JoinArgs &a,
                                      int lane) {
    __syncwarp();
    if (em.fill == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.counter[0], (unsigned long long)em.fill);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!a.count_only) {
        for (uint32_t i = lane; i < em.fill; i += 32) {
            uint64_t pos = base + i;
            if (pos < a.cap) a.out[pos] = ws.emit[i];
        }
    }
    __syncwarp();
    em.fill = 0;
}

// Stages the pairs of this lane's candidates for one query.
// n[c] = number of pairs (0, 1 or 2) for candidate slot c.
__device__ __forceinline__ void emit_pairs(Emitter &em, const WarpSmem &ws, const JoinArgs &a,
                                           int lane, uint32_t qid, const uint32_t *cid,
                                           const uint32_t *n) {
    uint32_t mine = 0;
#pragma unroll
    for (int c = 0; c < kCPL; ++c) mine += n[c];
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    if (em.fill + total > (uint32_t)a.eb) flush(em, ws, a, lane);
    if (!a.count_only) {
        uint32_t pos = em.fill + incl - mine;
#pragma unroll
        for (int c = 0; c < kCPL; ++c) {
            if (n[c] >= 1) ws.emit[pos++] = make_uint2(qid, cid[c]);
            if (n[c] == 2) ws.emit[pos++] = make_uint2(cid[c], qid);
        }
    }
    em.fill += total;
}

// Issues the bulk copies that bring flat candidates [k0, k1) of the item
// into a chunk buffer.  `rcur` is the first range that may overlap k0.
__device__ __forceinline__ void issue_chunk(const WarpSmem &ws, int buf, uint32_t k0, uint32_t k1,
                                            uint32_t nranges, uint32_t &rcur,
                                            const unsigned char *__restrict__ rec, uint32_t rsb,
                                            int lane) {
    while (rcur < nranges && ws.ranges[rcur].y <= k0) ++rcur;
    // earlier generic-proxy reads of this buffer precede the async-proxy writes
    fence_proxy_async_smem();
    if (lane == 0) mbar_arrive_expect_tx(&ws.bar[buf], (k1 - k0) * rsb);
    __syncwarp();
    for (uint32_t r0 = rcur; r0 < nranges; r0 += 32) {
        const uint32_t r = r0 + lane;
        bool starts_before = false;
        if (r < nranges) {
            const uint2 rg = ws.ranges[r];
            const uint32_t fs = (r == 0) ? 0u : ws.ranges[r - 1].y;
            const uint32_t fe = rg.y;
            starts_before = fs < k1;
            if (starts_before && fe > k0) {
                const uint32_t lo = fs > k0 ? fs : k0;
                const uint32_t hi = fe < k1 ? fe : k1;
                bulk_g2s(ws.buf[buf] + (size_t)(lo - k0) * rsb,
                         rec + (size_t)(rg.x + (lo - fs)) * rsb, (hi - lo) * rsb, &ws.bar[buf]);
            }
        }
        if (__ballot_sync(0xffffffffu, starts_before) != 0xffffffffu) break;
    }
}

// ---------------------------------------------------------------- the kernel

template <int D, bool F32, bool UNI>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2) join_kernel(const JoinArgs a,
                                                                     const uint32_t *counts) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const WarpSmem ws = carve(smem, a, warp);
    typedef typename std::conditional<F32, float, double>::type T;
    const uint32_t rsb = (uint32_t)a.rs * sizeof(T);
    const unsigned char *rec = F32 ? reinterpret_cast<const unsigned char *>(a.rec32)
                                   : reinterpret_cast<const unsigned char *>(a.rec64);

    if (lane == 0) {
        mbar_init(&ws.bar[0], 1);
        mbar_init(&ws.bar[1], 1);
    }
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t phase = 0;  // bit b: parity of the next completion of buffer b

    // counts[0] = |G|, counts[1] = number of work items (device-side, so the
    // launch needs no read-back)
    const uint32_t n_cells = counts[0];
    uint32_t item_end = a.item_end;
    if (counts[1] < item_end) item_end = counts[1];

    Emitter em;
    unsigned long long evals = 0, rechecks = 0;
    bool failed = false;

    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(a.work, (uint32_t)a.grab);
        first = __shfl_sync(0xffffffffu, first, 0);
        // sampled launches take every item_stride-th item
        const uint64_t f64 = (uint64_t)a.item_begin + (uint64_t)first * a.item_stride;
        if (f64 >= item_end) break;
        for (uint32_t g = 0; g < (uint32_t)a.grab && !failed; ++g) {
            const uint64_t item64 = f64 + (uint64_t)g * a.item_stride;
            if (item64 >= item_end) break;
            const uint2 it = a.items[item64];
            const uint32_t h = it.x;
            const uint32_t cbeg = a.G[h], cend = a.G[h + 1];
            const uint32_t home_len = cend - cbeg;
            const uint32_t q0 = cbeg + it.y * kQueryBlock;
            const uint32_t nq = min((uint32_t)kQueryBlock, cend - q0);

            // query records into shared memory
            {
                const uint32_t words = rsb / 16;
                const uint4 *src = reinterpret_cast<const uint4 *>(rec + (size_t)q0 * rsb);
                uint4 *dst = reinterpret_cast<uint4 *>(ws.q);
                for (uint32_t i = lane; i < nq * words; i += 32) dst[i] = src[i];
            }

            // cell coordinates and UNICOMP parity mask
            int32_t c[D];
            uint32_t odd = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                c[j] = a.cc[(uint64_t)h * D + j];
                odd |= ((uint32_t)c[j] & 1u) << j;
            }

            // 1. candidate ranges
            uint32_t nranges = 0, K = 0;
            for (int t0 = 0; t0 < a.n_templates; t0 += 32) {
                const int t = t0 + lane;
                uint32_t beg = 0, len = 0;
                int32_t xlo, xhi, b[D];
                if (t < a.n_templates && row_of<D, UNI>(t, c, odd, a, xlo, xhi, b)) {
                    uint64_t base = 0;
#pragma unroll
                    for (int j = 1; j < D; ++j) base += (uint64_t)b[j] * a.stride[j];
                    const uint64_t id_lo = base + (uint64_t)xlo, id_hi = base + (uint64_t)xhi;
                    uint32_t e;
                    if (a.dense) {
                        beg = __ldg(&a.lut[id_lo]);
                        e = __ldg(&a.lut[id_hi + 1]);
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
                    uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (len > 0) {
                    const uint32_t pos = nranges + __popc(nz & ((1u << lane) - 1u));
                    ws.ranges[pos] = make_uint2(beg, K + incl);
                }
                nranges += __popc(nz);
                K += __shfl_sync(0xffffffffu, incl, 31);
            }
            __syncwarp();

            // algorithmic evaluations of this item
            if (lane == 0) {
                if (UNI) {
                    const uint64_t ql0 = (uint64_t)it.y * kQueryBlock;
                    evals += (uint64_t)nq * (K - home_len) + (uint64_t)nq * (home_len - 1) -
                             (uint64_t)nq * ql0 - (uint64_t)nq * (nq - 1) / 2;
                } else {
                    evals += (uint64_t)nq * K;
                }
            }

            // 2-4. stream the candidates through the chunk buffers
            const uint32_t nchunks = (K + kChunk - 1) / kChunk;
            uint32_t rcur = 0;
            issue_chunk(ws, 0, 0, min(K, (uint32_t)kChunk), nranges, rcur, rec, rsb, lane);
            for (uint32_t ch = 0; ch < nchunks; ++ch) {
                const int bsel = ch & 1;
                if (ch + 1 < nchunks) {
                    const uint32_t k0 = (ch + 1) * kChunk;
                    issue_chunk(ws, bsel ^ 1, k0, min(K, k0 + kChunk), nranges, rcur, rec, rsb,
                                lane);
                }
                if (!mbar_wait_bounded(&ws.bar[bsel], (phase >> bsel) & 1u, a.timeout_ns)) {
                    failed = true;
                    if (lane == 0) atomicOr(a.error, kErrTimeout);
                    // let the other buffer's copies land before leaving
                    if (ch + 1 < nchunks)
                        (void)mbar_wait_bounded(&ws.bar[bsel ^ 1], (phase >> (bsel ^ 1)) & 1u,
                                                a.timeout_ns);
                    break;
                }
                phase ^= 1u << bsel;

                const uint32_t kb = ch * kChunk;
                const uint32_t clen = min((uint32_t)kChunk, K - kb);
                const T *cb = reinterpret_cast<const T *>(ws.buf[bsel]);
                const T *qb = reinterpret_cast<const T *>(ws.q);
                const bool home_chunk = UNI && kb < home_len;
                const uint32_t ql_base = it.y * kQueryBlock;

                // this lane's candidates
                T y[kCPL][D];
                uint32_t cid[kCPL];
                uint32_t kflat[kCPL];
#pragma unroll
                for (int s = 0; s < kCPL; ++s) {
                    const uint32_t slot = lane + 32 * s;
                    kflat[s] = kb + slot;
                    if (slot < clen) {
                        const T *r = cb + (size_t)slot * a.rs;
#pragma unroll
                        for (int j = 0; j < D; ++j) y[s][j] = r[j];
                        if (F32)
                            cid[s] = __float_as_uint((float)r[D]);
                        else
                            cid[s] = (uint32_t)__double_as_longlong((double)r[D]);
                    } else {
#pragma unroll
                        for (int j = 0; j < D; ++j) y[s][j] = (T)INFINITY;
                        cid[s] = 0xffffffffu;
                    }
                }

                if (F32) {
                    f2_t cx[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) cx[j] = f2_pack((float)y[0][j], (float)y[1][j]);
                    const float lo32 = a.lo32, hi32 = a.hi32;
                    for (uint32_t qi = 0; qi < nq; ++qi) {
                        const float *qr = reinterpret_cast<const float *>(qb) + (size_t)qi * a.rs;
                        float qv[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) qv[j] = qr[j];
                        f2_t t = f2_sub(cx[0], f2_pack(qv[0], qv[0]));
                        f2_t s2 = f2_mul(t, t);
#pragma unroll
                        for (int j = 1; j < D; ++j) {
                            t = f2_sub(cx[j], f2_pack(qv[j], qv[j]));
                            s2 = f2_fma(t, t, s2);
                        }
                        float sv[2];
                        f2_unpack(s2, sv[0], sv[1]);
                        bool maybe[kCPL];
#pragma unroll
                        for (int s = 0; s < kCPL; ++s) maybe[s] = sv[s] <= hi32;
                        if (home_chunk) {
                            const uint32_t ql = ql_base + qi;
#pragma unroll
                            for (int s = 0; s < kCPL; ++s)
                                if (kflat[s] < home_len && kflat[s] < ql) maybe[s] = false;
                        }
                        if (!__any_sync(0xffffffffu, maybe[0] | maybe[1])) continue;
                        const uint32_t qid = __float_as_uint(qr[D]);
                        uint32_t npairs[kCPL];
#pragma unroll
                        for (int s = 0; s < kCPL; ++s) {
                            bool hit = maybe[s];
                            const bool self = home_chunk && kflat[s] == ql_base + qi;
                            if (hit && !self && sv[s] > lo32) {
                                ++rechecks;
                                hit = exact_member<D>(a.pts + (size_t)qid * D,
                                                      a.pts + (size_t)cid[s] * D, a.E2);
                            }
                            npairs[s] = hit ? ((UNI && !self) ? 2u : 1u) : 0u;
                        }
                        emit_pairs(em, ws, a, lane, qid, cid, npairs);
                    }
                } else {
                    for (uint32_t qi = 0; qi < nq; ++qi) {
                        const double *qr =
                            reinterpret_cast<const double *>(qb) + (size_t)qi * a.rs;
                        double qv[D];
#pragma unroll
                        for (int j = 0; j < D; ++j) qv[j] = qr[j];
                        bool hitv[kCPL];
#pragma unroll
                        for (int s = 0; s < kCPL; ++s) {
                            double sd = 0.0;
#pragma unroll
                            for (int j = 0; j < D; ++j) {
                                double t = __dsub_rn(qv[j], (double)y[s][j]);
                                sd = __dadd_rn(sd, __dmul_rn(t, t));
                            }
                            hitv[s] = (sd <= a.E2) && cid[s] != 0xffffffffu;
                        }
                        if (home_chunk) {
                            const uint32_t ql = ql_base + qi;
#pragma unroll
                            for (int s = 0; s < kCPL; ++s)
                                if (kflat[s] < home_len && kflat[s] < ql) hitv[s] = false;
                        }
                        if (!__any_sync(0xffffffffu, hitv[0] | hitv[1])) continue;
                        const uint32_t qid = (uint32_t)__double_as_longlong(qr[D]);
                        uint32_t npairs[kCPL];
#pragma unroll
                        for (int s = 0; s < kCPL; ++s) {
                            const bool self = home_chunk && kflat[s] == ql_base + qi;
                            npairs[s] = hitv[s] ? ((UNI && !self) ? 2u : 1u) : 0u;
                        }
                        emit_pairs(em, ws, a, lane, qid, cid, npairs);
                    }
                }
                __syncwarp();
            }
            __syncwarp();
        }
        if (failed) break;
    }
    flush(em, ws, a, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
    if (lane == 0) {
        if (evals) atomicAdd(&a.counter[1], evals);
        if (rechecks) atomicAdd(&a.counter[2], rechecks);
    }
}

typedef void (*KernelFn)(const JoinArgs, const uint32_t *);

template <int D>
KernelFn pick(bool f32, bool uni) {
    if (f32) return uni ? join_kernel<D, true, true> : join_kernel<D, true, false>;
    return uni ? join_kernel<D, false, true> : join_kernel<D, false, false>;
}

KernelFn pick_kernel(int d, bool f32, bool uni) {
    switch (d) {
        case 1: return pick<1>(f32, uni);
        case 2: return pick<2>(f32, uni);
        case 3: return pick<3>(f32, uni);
        case 4: return pick<4>(f32, uni);
        case 5: return pick<5>(f32, uni);
        case 6: return pick<6>(f32, uni);
        case 7: return pick<7>(f32, uni);
        case 8: return pick<8>(f32, uni);
        default: return nullptr;
    }
}

inline int round16(int x) { return (x + 15) & ~15; }

}  // namespace

int n_templates(int d, bool uni) {
    int p = 1;
    for (int j = 1; j < d; ++j) p *= 3;
    return uni ? p + 2 : p;
}

sj_status launch_join(Error &err, const Index &ix, const JoinLaunch &cfg, uint32_t item_begin,
                      uint32_t item_end, uint2 *out, uint64_t cap,
                      unsigned long long *d_counter, uint32_t *d_work, uint32_t *d_error,
                      int count_only, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    const Geometry &g = ix.g;
    const int d = g.d;
    const bool f32 = cfg.prec_fp32 && g.fp32_ok;
    const bool uni = cfg.unicomp != 0;
    if (!f32 && !ix.rec64.p) return fail(err, SJ_EINVAL, "FP64 records missing");
    JoinArgs a;
    memset(&a, 0, sizeof(a));
    a.rec32 = static_cast<const float *>(ix.rec32.p);
    a.rec64 = static_cast<const double *>(ix.rec64.p);
    a.pts = static_cast<const double *>(ix.pts.p);
    a.G = static_cast<const uint32_t *>(ix.G.p);
    a.B = static_cast<const uint64_t *>(ix.B.p);
    a.cc = static_cast<const int32_t *>(ix.cc.p);
    a.M = static_cast<const uint32_t *>(ix.M.p);
    a.lut = static_cast<const uint32_t *>(ix.lut.p);
    a.items = static_cast<const uint2 *>(ix.items.p);
    a.item_begin = item_begin;
    a.item_end = item_end;
    a.item_stride = cfg.item_stride > 0 ? cfg.item_stride : 1;
    a.mwords = ix.mwords;
    a.dense = ix.dense;
    a.rs = f32 ? ix.rs32 : ix.rs64;
    a.n_templates = n_templates(d, uni);
    for (int j = 0; j < d; ++j) {
        a.ng[j] = (int32_t)g.ng[j];
        a.stride[j] = g.stride[j];
    }
    a.lo32 = g.lo32;
    a.hi32 = g.hi32;
    a.E2 = g.E2;
    a.out = out;
    a.cap = cap;
    a.counter = d_counter;
    a.work = d_work;
    a.error = d_error;
    a.count_only = count_only;
    a.grab = cfg.grab > 0 ? cfg.grab : 1;
    const int esz = f32 ? 4 : 8;
    const int rsb = a.rs * esz;
    a.sm_ranges = round16(a.n_templates * (int)sizeof(uint2));
    a.sm_queries = round16(kQueryBlock * rsb);
    a.sm_chunk = round16(kChunk * rsb);
    a.eb = kEmit;
    a.sm_emit = round16(kEmit * (int)sizeof(uint2));
    a.sm_warp = 16 + a.sm_ranges + a.sm_queries + 2 * a.sm_chunk + a.sm_emit;
    a.cb = kChunk;
    a.timeout_ns = 2000000000ull;

    KernelFn fn = pick_kernel(d, f32, uni);
    if (!fn) return fail(err, SJ_EINVAL, "unsupported dimension");
    const size_t smem = (size_t)a.sm_warp * kWarpsPerBlock;
    SJ_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0;
    SJ_CUDA_TRY(cudaGetDevice(&dev));
    int per_sm = 0;
    SJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWarpsPerBlock * 32, smem));
    if (per_sm < 1) return fail(err, SJ_EINVAL, "join kernel does not fit on an SM");
    int blocks = cfg.blocks > 0 ? cfg.blocks : per_sm * sm_count(dev);
    if (item_end <= item_begin) blocks = 1;
    SJ_CUDA_TRY(cudaMemsetAsync(d_work, 0, sizeof(uint32_t), s));
    if (ev0) SJ_CUDA_TRY(cudaEventRecord(ev0, s));
    fn<<<blocks, kWarpsPerBlock * 32, smem, s>>>(a, n_items_dev(ix) - 1); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    if (ev1) SJ_CUDA_TRY(cudaEventRecord(ev1, s));
    return SJ_OK;
}

}  // namespace sj
