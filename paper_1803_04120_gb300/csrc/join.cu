// join.cu -- persistent search-and-refine kernel (Section IV-D, IV-E, V-B).
//
// Work decomposition.  A work item is (non-empty cell h, block of up to 32
// of its points).  Items are taken from a global cursor by whole warps, so
// heavy cells are spread over many warps.  Per item a warp
//   1. builds the candidate ranges: the adjacent cells the query cell must
//      search (Section IV-D), chosen by UNICOMP (Section V-B) or all 3^n of
//      them (Algorithm 1).  Cells adjacent along dimension 1 have consecutive
//      linear ids, so a "row" of up to three cells that agree in dimensions
//      2..n is one contiguous range of the cell-ordered records; a row is
//      skipped when M_j marks one of its fixed coordinates as empty, and is
//      looked up with two loads of the dense table or two binary searches of
//      B.  The home cell is range 0.
//   2. stages its query points in shared memory, already transformed for the
//      distance evaluation (see below).
//   3. streams the candidates through a ring of NBUF shared-memory chunk
//      buffers: each range piece of a chunk is one cp.async.bulk copy of
//      16-byte aligned records, completing on the slot's mbarrier.  The
//      producer side of the warp runs up to NBUF chunks ahead of the
//      consumer side and crosses into the next work item (two item slots),
//      so copy latency is hidden also when items are small.
//   4. compares: lanes own CPL candidates each, the queries are broadcast
//      from shared memory.
//        FP32 mode: coordinates relative to the home cell's centre,
//        z = fl32(y - o), and s = |z_p|^2 + |z_q|^2 - 2 z_p . z_q evaluated
//        as one add and d fused multiply-adds on packed f32x2 pairs (two
//        candidates per instruction).  s is compared with the proven margin
//        [lo32, hi32] computed on the host (margin.cu): per candidate slot
//        each lane keeps a 32-bit mask of the queries within hi32, and the
//        largest value among its hits.  Only when that maximum exceeds
//        lo32 (a hit in the band: a few in 1e4) are the chunk's hits
//        re-evaluated to find the band ones, which the exact FP64
//        predicate decides, in a warp-uniform branch around a non-inlined
//        function so that the slow FP64 pipe of GB300 sees only the real
//        rechecks.
//        FP64 mode: the exact predicate for every candidate.
//   5. emits: FP32 mode under UNICOMP: the self-pair of every query once
//      per item, then each hit (p, q) gives (p, q) and (q, p), and in the
//      home cell only candidates after the query's own position count (the
//      masks are cleared with bit operations); without UNICOMP each hit
//      gives (p, q), the self-pair included.  Pairs are staged per warp in
//      shared memory in a few rounds per chunk, one warp scan each.  FP64
//      mode: per query, ballot + popc offsets, the self-pair once.  Staged
//      pairs are written out in coalesced blocks after one atomic
//      reservation per flush.
// Waits on mbarriers are bounded by a time limit; on expiry the warp records
// an error bit, waits (bounded) for its copies in flight and leaves.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "join_dev.cuh"

namespace sj {

namespace {

// The kernel is latency-bound (dependent shared-memory loads and ALU chains
// per warp), so the per-warp shared memory and registers are sized for
// resident warps: measured on GB300 with 2,000,000 uniform points.
// Candidates per lane by dimension and precision (chunk = 32 * CPL): four
// at d >= 5, where each chunk's loads are shared by the most comparisons;
// two below, where the smaller registers and ring let three blocks reside
// (d = 4: 1.28 ms against 1.35 ms with four; d = 5: 2.63 against 2.41).
__host__ __device__ constexpr int cpl_for(int d, bool f32) { return f32 ? (d <= 4 ? 2 : 4) : 2; }
// FP32 strides in floats (the host's index and launch set the same): a
// point record x_0 .. x_{d-1}, id padded to 16 bytes; a staged query record
// m_0 .. m_{d-1}, pp, id padded to 16 bytes.  Compile-time in the kernel.
__host__ __device__ constexpr int rs32_for(int d) { return (d + 1 + 3) / 4 * 4; }
__host__ __device__ constexpr int qrs32_for(int d) { return (d + 2 + 3) & ~3; }
// FP64 strides in doubles: a point record and a staged query record are
// both x_0 .. x_{d-1}, id padded to 16 bytes.
__host__ __device__ constexpr int rs64_for(int d) { return (d + 1 + 1) / 2 * 2; }
__host__ __device__ constexpr int rs_for(int d, bool f32) { return f32 ? rs32_for(d) : rs64_for(d); }
// Default depth of the chunk ring (a launch may choose another).
__host__ __device__ constexpr int nbuf_for(int d, bool f32) { return (f32 && d >= 4) ? 2 : 4; }
// Staged pairs per warp: many pairs per chunk at low d want a large staging
// area (every flush waits for one global atomic reservation; clustered 3-D
// data: 27.7 ms with 256 against 13.1 ms with 512); at higher d a smaller
// one leaves room for warps (the tuner may still choose more).
__host__ __device__ constexpr int emit_for(int d, bool f32) { return (f32 && d >= 4) ? 256 : 512; }
// Item slots per warp: at d >= 4 an item spans tens of chunks, so
// preparing the next item ahead buys little and its shared memory is worth
// more as resident warps.
__host__ __device__ constexpr int slots_for(int d, bool f32) { return (f32 && d >= 4) ? 1 : 2; }
// Minimum resident blocks of 256 threads the compiler sizes registers for.
__host__ __device__ constexpr int minb_for(int d, bool f32) { return f32 ? (d <= 2 ? 1 : (d <= 4 ? 3 : 2)) : 1; }

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
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
        if ((it & 15) == 15 && global_ns() - t0 > limit_ns) return false;
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

// The exact predicate of Section III in FP64: every operation rounded to
// nearest on its own, no contraction.  Kept out of line so that the FP64
// instructions run only for the pairs that need them.
__device__ __noinline__ bool exact_member_ni(const double *__restrict__ a,
                                             const double *__restrict__ b, int d, double E2) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = __dsub_rn(a[j], b[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s <= E2;
}

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

// The row-template table (entry format in join_dev.cuh).
constexpr int kTemplateEntries = 6576;   // sum over d = 1..8 of both tables
__device__ uint32_t g_templates[kTemplateEntries];

// Per-item header kept in shared memory (one per item slot).
struct ItemHdr {
    uint32_t h, qb, nq, home_len, K, nchunks, nranges, pad;
    float o[kMaxDim];
};

// Per-warp shared-memory carve-up.
struct WarpSmem {
    uint64_t *bar;            // one mbarrier per ring slot
    ItemHdr *hdr;             // [2]
    uint2 *ranges[2];         // (begin in cell order, flat end)
    unsigned char *q[2];      // query records
    unsigned char *ring;      // chunk buffers
    uint2 *emit;
};

__device__ __forceinline__ WarpSmem carve(unsigned char *base, const JoinArgs &a, int warp,
                                          int nbuf) {
    WarpSmem w;
    unsigned char *p = base + (size_t)warp * a.sm_warp;
    w.bar = reinterpret_cast<uint64_t *>(p);
    p += 64;
    // one or two item slots (the second lets the producer prepare the next
    // item while the consumer still works on the current one)
    const int two = a.slots > 1 ? 1 : 0;
    w.hdr = reinterpret_cast<ItemHdr *>(p);
    p += (1 + two) * sizeof(ItemHdr);
    w.ranges[0] = reinterpret_cast<uint2 *>(p);
    p += a.sm_ranges;
    w.ranges[1] = reinterpret_cast<uint2 *>(p - (two ? 0 : a.sm_ranges));
    p += two * a.sm_ranges;
    w.q[0] = p;
    p += a.sm_queries;
    w.q[1] = p - (two ? 0 : a.sm_queries);
    p += two * a.sm_queries;
    w.ring = p;
    p += (size_t)nbuf * a.sm_chunk;
    w.emit = reinterpret_cast<uint2 *>(p);
    return w;
}

// Warp-uniform state of the producer / consumer pipeline.
struct Pipe {
    uint32_t grab_pos, grab_end;   // work-cursor positions taken by this warp
    uint32_t issued, consumed;     // chunks
    uint32_t p_slot, c_slot;       // ring slots of the next issue / consume
    uint32_t c_phase;              // mbarrier phase parity of the next consume
    uint32_t prod_seq, cons_seq;   // item sequence numbers (slot = seq & smask)
    uint32_t p_chunk, c_chunk;
    uint32_t rcur;                 // producer's range cursor
    uint32_t fill;                 // staged pairs
    bool prod_done;
};

__device__ __forceinline__ void flush(Pipe &st, const WarpSmem &ws, const JoinArgs &a, int lane) {
    __syncwarp();
    if (st.fill == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.counter[0], (unsigned long long)st.fill);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!a.count_only) {
        // positions relative to the reservation, bounded by cap once
        uint2 *const out = a.out + base;
        const uint32_t n = a.cap > base ? (uint32_t)min((uint64_t)(a.cap - base), (uint64_t)st.fill) : 0u;
        for (uint32_t i = lane; i < n; i += 32) __stcs(&out[i], ws.emit[i]);
    }
    __syncwarp();
    st.fill = 0;
}

// Stages the pairs of candidate slot s of every lane for one query:
// npairs in {0, 1, 2}.  Offsets come from two ballots.
__device__ __forceinline__ void emit_slot(Pipe &st, const WarpSmem &ws, const JoinArgs &a, int lane,
                                          uint32_t qid, uint32_t cid, uint32_t npairs) {
    const unsigned m1 = __ballot_sync(0xffffffffu, npairs >= 1);
    if (m1 == 0) return;
    const unsigned m2 = __ballot_sync(0xffffffffu, npairs == 2);
    const unsigned lt = (1u << lane) - 1u;
    if (npairs && !a.count_only) {
        uint32_t pos = st.fill + __popc(m1 & lt) + __popc(m2 & lt);
        ws.emit[pos] = make_uint2(qid, cid);
        if (npairs == 2) ws.emit[pos + 1] = make_uint2(cid, qid);
    }
    st.fill += __popc(m1) + __popc(m2);
}

// Loads this lane's CPL candidates of a chunk (slot s = position lane + 32 s)
// from shared memory with 16-byte loads, moves them into the frame of the
// home cell centre o and packs them in pairs.  Slots past the chunk end get
// z = 0, |z|^2 = +inf (never a member) and id 0xffffffff.
// WRAP (cell-frame records): a candidate stored in the neighbouring
// four-cell frame is moved by k = -rint(z / (4 w32)) frame steps,
// z - 4 w32 k, which is exact.
template <int D, int CPL, bool WRAP>
__device__ __forceinline__ void load_candidates(const unsigned char *buf, int rs, uint32_t clen,
                                                int lane, const float *o_smem, float w4,
                                                float inv_w4, f2_t (*z)[D], f2_t *qq2,
                                                uint32_t *cid) {
    constexpr int V = (D + 1 + 3) / 4;    // float4 per record (rs = 4 V)
    float o[D];
#pragma unroll
    for (int j = 0; j < D; ++j) o[j] = o_smem[j];
#pragma unroll
    for (int cp = 0; cp < CPL / 2; ++cp) {
        float za[2][D], qs[2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = 2 * cp + h2;
            const uint32_t slot = lane + 32 * s;
            qs[h2] = INFINITY;
#pragma unroll
            for (int j = 0; j < D; ++j) za[h2][j] = 0.0f;
            cid[s] = 0xffffffffu;
            if (slot < clen) {
                const float4 *rr = reinterpret_cast<const float4 *>(buf + (size_t)slot * rs * 4);
                float r[4 * V];
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const float4 v = rr[k];
                    r[4 * k] = v.x;
                    r[4 * k + 1] = v.y;
                    r[4 * k + 2] = v.z;
                    r[4 * k + 3] = v.w;
                }
                float q2 = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float zz = __fsub_rn(r[j], o[j]);
                    if (WRAP) zz = __fmaf_rn(-w4, rintf(__fmul_rn(zz, inv_w4)), zz);
                    za[h2][j] = zz;
                    q2 = __fmaf_rn(zz, zz, q2);
                }
                qs[h2] = q2;
                cid[s] = __float_as_uint(r[D]);
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) z[cp][j] = f2_pack(za[0][j], za[1][j]);
        qq2[cp] = f2_pack(qs[0], qs[1]);
    }
}

// s32 for one staged query record against this lane's candidates:
// fl(|z_q|^2 + |z_p|^2) then d fused multiply-adds with m_j = -2 z_p,j;
// with SHIFT, fl(s32 + shift) (a packed pair added to both values).
template <int D, int NP, bool SHIFT = false>
__device__ __forceinline__ void eval_query(const float *qd, const f2_t (*z)[D], const f2_t *qq2,
                                           float *sv, f2_t shift = 0ull) {
    // record: m_0 .. m_{d-1}, pp, id (16-byte loads, broadcast to the warp)
    constexpr int V = (D + 2 + 3) / 4;
    float r[4 * V];
    const float4 *q4 = reinterpret_cast<const float4 *>(qd);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float4 v = q4[k];
        r[4 * k] = v.x;
        r[4 * k + 1] = v.y;
        r[4 * k + 2] = v.z;
        r[4 * k + 3] = v.w;
    }
    const f2_t pp = f2_pack(r[D], r[D]);
    f2_t acc[NP];
#pragma unroll
    for (int cp = 0; cp < NP; ++cp) acc[cp] = f2_add(qq2[cp], pp);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const f2_t mj = f2_pack(r[j], r[j]);
#pragma unroll
        for (int cp = 0; cp < NP; ++cp) acc[cp] = f2_fma(mj, z[cp][j], acc[cp]);
    }
#pragma unroll
    for (int cp = 0; cp < NP; ++cp) {
        if (SHIFT) acc[cp] = f2_add(acc[cp], shift);
        f2_unpack(acc[cp], sv[2 * cp], sv[2 * cp + 1]);
    }
}

// Takes the next work item for this warp; false when none is left.
__device__ __forceinline__ bool fetch_item(Pipe &st, const JoinArgs &a, uint32_t item_end,
                                           int lane, uint2 &it) {
    if (st.grab_pos == st.grab_end) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(a.work, (uint32_t)a.grab);
        first = __shfl_sync(0xffffffffu, first, 0);
        st.grab_pos = first;
        st.grab_end = first + a.grab;
    }
    const uint64_t item = (uint64_t)a.item_begin + (uint64_t)st.grab_pos * a.item_stride;
    if (item >= item_end) return false;
    ++st.grab_pos;
    it = a.items[item];
    return true;
}

// Builds ranges, header and staged queries of item `it` in item slot `sl`.
template <int D, bool F32, bool UNI>
__device__ __forceinline__ void prepare_item(const WarpSmem &ws, int sl, uint2 it,
                                             const JoinArgs &a, uint32_t n_cells, int lane,
                                             unsigned long long &evals) {
    typedef typename std::conditional<F32, float, double>::type T;
    const uint32_t rsb = (uint32_t)(rs_for(D, F32) * sizeof(T));
    // the query side: the item's cell and points (the candidate side is
    // read through a.lut / a.B / a.G and the ranges)
    const unsigned char *rec = F32 ? reinterpret_cast<const unsigned char *>(a.qrec32)
                                   : reinterpret_cast<const unsigned char *>(a.qrec64);
    const uint32_t h = it.x;
    const uint32_t cbeg = __ldg(&a.qG[h]), cend = __ldg(&a.qG[h + 1]);
    const uint32_t home_len = cend - cbeg;
    const uint32_t q0 = cbeg + it.y * kQueryBlock;
    const uint32_t nq = min((uint32_t)kQueryBlock, cend - q0);

    int32_t c[D];
    uint32_t odd = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        c[j] = __ldg(&a.qcc[(uint64_t)h * D + j]);
        odd |= ((uint32_t)c[j] & 1u) << j;
    }

    // candidate ranges
    uint2 *rt = ws.ranges[sl];
    uint32_t nranges, K;
    build_ranges<D, UNI>(c, odd, a, n_cells, lane, rt, nranges, K);

    // staged queries
    ItemHdr *hd = &ws.hdr[sl];
    if (F32) {
        float o[D];
#pragma unroll
        for (int j = 0; j < D; ++j)
            o[j] = ((float)(a.frame == SJ_FRAME_CELL ? (c[j] & 3) : c[j]) + 0.5f) * a.w32;
        if (lane < (int)nq) {
            const float *r = reinterpret_cast<const float *>(rec + (size_t)(q0 + lane) * rsb);
            float *qd = reinterpret_cast<float *>(ws.q[sl]) + (size_t)lane * qrs32_for(D);
            float pp = 0.0f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float z = __fsub_rn(r[j], o[j]);
                pp = __fmaf_rn(z, z, pp);
                const float m = -2.0f * z;
                qd[j] = m;
            }
            qd[D] = pp;
            qd[D + 1] = r[D];   // point id bits
        }
        if (lane < D) hd->o[lane] = o[lane];
    } else {
        if (lane < (int)nq) {
            const double *r = reinterpret_cast<const double *>(rec + (size_t)(q0 + lane) * rsb);
            double *qd = reinterpret_cast<double *>(ws.q[sl]) + (size_t)lane * rs64_for(D);
#pragma unroll
            for (int j = 0; j <= D; ++j) qd[j] = r[j];
        }
    }
    if (lane == 0) {
        hd->h = h;
        hd->qb = it.y;
        hd->nq = nq;
        hd->home_len = home_len;
        hd->K = K;
        hd->nchunks = (K + 32 * cpl_for(D, F32) - 1) / (32 * cpl_for(D, F32));
        hd->nranges = nranges;
        // algorithmic evaluations of this item
        if (UNI) {
            const uint64_t ql0 = (uint64_t)it.y * kQueryBlock;
            evals += (uint64_t)nq * (K - home_len) + (uint64_t)nq * (home_len - 1) -
                     (uint64_t)nq * ql0 - (uint64_t)nq * (nq - 1) / 2;
        } else {
            evals += (uint64_t)nq * K;
        }
    }
    __syncwarp();
}

// Issues the bulk copies of chunk `ch` of the item in slot `sl` into ring
// slot `r`.
template <int CB>
__device__ __forceinline__ void issue_chunk(const WarpSmem &ws, int sl, uint32_t ch, int r,
                                            uint32_t &rcur, const unsigned char *__restrict__ rec,
                                            uint32_t rsb, int lane, int sm_chunk) {
    const ItemHdr *hd = &ws.hdr[sl];
    const uint32_t K = hd->K, nranges = hd->nranges;
    const uint2 *rt = ws.ranges[sl];
    const uint32_t k0 = ch * CB;
    const uint32_t k1 = min(K, k0 + CB);
    unsigned char *buf = ws.ring + (size_t)r * sm_chunk;
    // earlier generic-proxy reads of this buffer precede the async-proxy writes
    fence_proxy_async_smem();
    if (lane == 0) mbar_arrive_expect_tx(&ws.bar[r], (k1 - k0) * rsb);
    __syncwarp();
    // rcur is the first range that ends after k0 (ranges end at increasing
    // flat positions); lane l looks at range rcur + l, and the ranges that
    // end by k1 are skipped for the next chunk with one ballot
    for (uint32_t r0 = rcur;; r0 += 32) {
        const uint32_t rr = r0 + lane;
        const bool valid = rr < nranges;
        const uint2 rg = valid ? rt[rr] : make_uint2(0u, 0xffffffffu);
        uint32_t fs = __shfl_up_sync(0xffffffffu, rg.y, 1);
        if (lane == 0) fs = rr == 0 ? 0u : rt[rr - 1].y;
        const uint32_t fe = rg.y;
        if (valid && fs < k1 && fe > k0) {
            const uint32_t lo = fs > k0 ? fs : k0;
            const uint32_t hi = fe < k1 ? fe : k1;
            bulk_g2s(buf + (size_t)(lo - k0) * rsb, rec + (size_t)(rg.x + (lo - fs)) * rsb,
                     (hi - lo) * rsb, &ws.bar[r]);
        }
        const unsigned done = __ballot_sync(0xffffffffu, valid && fe <= k1);
        rcur = r0 + __popc(done);
        // all 32 ranges end by k1: the chunk may cover more, look at the next 32
        if (done != 0xffffffffu) break;
    }
}

// Chunks with at least this many pairs write them straight to the output.
constexpr uint32_t kDirectPairs = 128;

// Writes up to c hits of this lane (the lowest query bits of the first
// non-empty candidate slots, cleared as they go) at dst[base ...] in
// (t, lane) order: at step t the pairs (p, q) of the active lanes, then
// their (q, p) under UNICOMP.  Lane l holds the id of query l in qid_l; the
// query id of a hit comes by shuffle.  Global destinations are bounded by
// cap.  Positions are kept relative to base in 32 bits (a chunk holds at
// most 2 * 32 * 32 * CPL pairs).
template <int CPL, bool UNI, bool GLOBAL>
__device__ __forceinline__ void put_hits(uint32_t (&m)[CPL], const uint32_t (&cid)[CPL],
                                         uint32_t qid_l, uint32_t c, uint64_t base, uint2 *dst,
                                         uint64_t cap, int lane) {
    constexpr uint32_t kPP = UNI ? 2u : 1u;
    const unsigned lt = (1u << lane) - 1u;
    uint2 *const out = dst + base;
    // pairs that still fit below cap, from base on
    const uint32_t room =
        GLOBAL ? (uint32_t)(cap > base ? min(cap - base, (uint64_t)0xffffffffu) : 0ull) : 0xffffffffu;
    uint32_t rel = 0;
    for (uint32_t t = 0;; ++t) {
        const bool act = t < c;
        const unsigned bm = __ballot_sync(0xffffffffu, act);
        if (!bm) break;
        const uint32_t nb = __popc(bm);
        // the lane's next hit: first non-empty slot, lowest query bit
        uint32_t q = 0, cand = 0;
        bool found = false;
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            const bool take = act && !found && m[s] != 0;
            if (take) {
                q = __ffs(m[s]) - 1;
                m[s] &= m[s] - 1;
                cand = cid[s];
            }
            found |= take;
        }
        const uint32_t qid = __shfl_sync(0xffffffffu, qid_l, q);
        if (act) {
            const uint32_t p = rel + __popc(bm & lt);
            if (GLOBAL) {
                // streaming stores: the pairs are never read back, so they
                // should not displace the candidate records from L2
                if (p < room) __stcs(&out[p], make_uint2(qid, cand));
                if (UNI && p + nb < room) __stcs(&out[p + nb], make_uint2(cand, qid));
            } else {
                out[p] = make_uint2(qid, cand);
                if (UNI) out[p + nb] = make_uint2(cand, qid);
            }
        }
        rel += kPP * nb;
    }
}

// Compares chunk `ch` (in ring slot r) of the item in slot `sl` with the
// item's queries and stages the pairs found.  FR: the FP32 record frame,
// 0 grid, 1 cell, 2 read from the arguments at run time (multi-join).
template <int D, bool F32, bool UNI, int FR>
__device__ __forceinline__ void consume_chunk(Pipe &st, const WarpSmem &ws, int sl, uint32_t ch,
                                              int r, const JoinArgs &a, int lane,
                                              unsigned long long &rechecks) {
    constexpr int CPL = cpl_for(D, F32);
    constexpr int CB = 32 * CPL;
    const ItemHdr *hd = &ws.hdr[sl];
    const uint32_t K = hd->K, nq = hd->nq, home_len = hd->home_len;
    const uint32_t kb = ch * CB;
    const uint32_t clen = min((uint32_t)CB, K - kb);
    const bool home_chunk = UNI && kb < home_len;
    const uint32_t ql_base = hd->qb * kQueryBlock;
    const unsigned char *buf =
        ws.ring + (size_t)r * ((CB * rs_for(D, F32) * (F32 ? 4 : 8) + 15) & ~15);

    if (F32) {
        constexpr int NP = CPL / 2;
        constexpr int QRS = qrs32_for(D), RS = rs32_for(D);
        const float hi32 = a.hi32, lo32 = a.lo32;
        f2_t z[NP][D], qq2[NP];
        uint32_t cid[CPL];
        if (FR == 2 ? a.frame == SJ_FRAME_CELL : FR == 1)
            load_candidates<D, CPL, true>(buf, RS, clen, lane, hd->o, a.w4, a.inv_w4, z, qq2, cid);
        else
            load_candidates<D, CPL, false>(buf, RS, clen, lane, hd->o, a.w4, a.inv_w4, z, qq2, cid);
        const float *qbase = reinterpret_cast<const float *>(ws.q[sl]);
        if (UNI && ch == 0) {
            // UNICOMP: the item's self-pairs, one per query point; every
            // other hit then stands for both (p, q) and (q, p).  (The full
            // search meets the query itself as an ordinary hit.)
            if (st.fill + nq > (uint32_t)a.eb) flush(st, ws, a, lane);
            if (!a.count_only && lane < (int)nq) {
                const uint32_t qid = __float_as_uint(qbase[(size_t)lane * QRS + D + 1]);
                ws.emit[st.fill + lane] = make_uint2(qid, qid);
            }
            st.fill += nq;
        }
        // 1. comparison: bit qi of m[s] = candidate slot s is within hi32 of
        //    query qi.  Each value is compared through dv = s32 - h with h
        //    the float just above hi32 (two packed subtractions per query):
        //    the sign of an IEEE difference is exact, so s32 <= hi32 iff dv
        //    is negative, and one funnel shift moves that sign bit into the
        //    mask (queries taken from the last to the first, so that query
        //    qi ends at bit qi).  Near the threshold dv is exact (Sterbenz),
        //    so a hit lies in the band above lo32 iff dv > lo32 - h, which
        //    for negative floats is an integer comparison of their bits: mn,
        //    the smallest bit pattern, tells whether the lane has such a hit
        //    (rare: a few in 1e4 hits).  Non-hits have non-negative dv and
        //    bit patterns above every hit's.
        uint32_t m[CPL], b[CPL];
#pragma unroll
        for (int s = 0; s < CPL; ++s) m[s] = b[s] = 0u;
        const float h1 = __int_as_float(__float_as_int(hi32) + 1);
        const f2_t mh = f2_pack(-h1, -h1);
        int mn = 0x7fffffff;
        for (int qi = (int)nq - 1; qi >= 0; --qi) {
            float sv[CPL];
            eval_query<D, NP, true>(qbase + (size_t)qi * QRS, z, qq2, sv, mh);
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                m[s] = __funnelshift_l(__float_as_uint(sv[s]), m[s], 1);
                mn = min(mn, __float_as_int(sv[s]));
            }
        }
        uint32_t any = 0;
#pragma unroll
        for (int s = 0; s < CPL; ++s) any |= m[s];
        if (!__any_sync(0xffffffffu, any)) return;
        // 2. UNICOMP home cell (range 0): only candidates after the query's
        //    own position count
        if (home_chunk) {
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                const uint32_t k = kb + lane + 32 * s;
                if (k < home_len) {
                    const uint32_t r = k > ql_base ? k - ql_base : 0u;
                    m[s] &= r >= 32 ? 0xffffffffu : ((1u << r) - 1u);
                }
            }
        }
        // 3. band: values above lo32 are decided by the exact FP64
        //    predicate.  Only in a chunk where some hit lies in the band are
        //    the hits re-evaluated to find which ones
        if (__any_sync(0xffffffffu, mn < __float_as_int(lo32 - h1))) {
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                uint32_t w = m[s];
                while (w) {
                    const uint32_t q = __ffs(w) - 1;
                    w &= w - 1;
                    float sv2[2];
                    eval_query<D, 1>(qbase + (size_t)q * QRS, &z[s >> 1], &qq2[s >> 1], sv2);
                    if (sv2[s & 1] > lo32) b[s] |= 1u << q;
                }
            }
        }
        uint32_t band = 0;
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            b[s] &= m[s];
            band |= b[s];
        }
        if (__any_sync(0xffffffffu, band)) {
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                uint32_t w = b[s];
                while (w) {
                    const uint32_t q = __ffs(w) - 1;
                    w &= w - 1;
                    ++rechecks;
                    const uint32_t qid = __float_as_uint(qbase[(size_t)q * QRS + D + 1]);
                    if (!exact_member_ni(a.qpts + (size_t)qid * D, a.pts + (size_t)cid[s] * D, D, a.E2))
                        m[s] &= ~(1u << q);
                }
            }
        }
        // 4. emission (the order of pairs in the output is free).  A chunk
        //    with many pairs reserves its output once and writes it straight
        //    to global memory in (t, lane) order: the t-th hit of every lane
        //    that has one goes to consecutive slots, so each store
        //    instruction writes consecutive words (coalesced).  A chunk with
        //    few pairs is staged in shared memory, each lane at its prefix
        //    position, so that the same-address reservations stay rare (one
        //    per flush of the staging area).
        constexpr uint32_t kPP = UNI ? 2u : 1u;
        uint32_t left = 0;
#pragma unroll
        for (int s = 0; s < CPL; ++s) left += __popc(m[s]);
        const uint32_t hits = __reduce_add_sync(0xffffffffu, left);
        if (hits == 0) return;
        if (hits * kPP >= kDirectPairs) {
            const uint32_t qid_l =
                lane < (int)nq ? __float_as_uint(qbase[(size_t)lane * QRS + D + 1]) : 0u;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&a.counter[0], (unsigned long long)hits * kPP);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (!a.count_only)
                put_hits<CPL, UNI, true>(m, cid, qid_l, left, base, a.out, a.cap, lane);
            return;
        }
        // fewer than kDirectPairs pairs: staged, each lane writing its own
        // hits at its exclusive prefix position (one warp scan)
        uint32_t incl = left;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = hits * kPP;
        if (st.fill + total > (uint32_t)a.eb) flush(st, ws, a, lane);
        if (!a.count_only) {
            uint32_t pos = st.fill + kPP * (incl - left);
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                uint32_t w = m[s];
                while (w) {
                    const uint32_t q = __ffs(w) - 1;
                    w &= w - 1;
                    const uint32_t qid = __float_as_uint(qbase[(size_t)q * QRS + D + 1]);
                    ws.emit[pos] = make_uint2(qid, cid[s]);
                    if (UNI) ws.emit[pos + 1] = make_uint2(cid[s], qid);
                    pos += kPP;
                }
            }
        }
        st.fill += total;
    } else {
        double y[CPL][D];
        uint32_t cid[CPL];
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            const uint32_t slot = lane + 32 * s;
            cid[s] = 0xffffffffu;
#pragma unroll
            for (int j = 0; j < D; ++j) y[s][j] = 0.0;
            if (slot < clen) {
                const double *rr = reinterpret_cast<const double *>(buf + (size_t)slot * rs64_for(D) * 8);
#pragma unroll
                for (int j = 0; j < D; ++j) y[s][j] = rr[j];
                cid[s] = (uint32_t)__double_as_longlong(rr[D]);
            }
        }
        const double *qbase = reinterpret_cast<const double *>(ws.q[sl]);
        for (uint32_t qi = 0; qi < nq; ++qi) {
            const double *qd = qbase + (size_t)qi * rs64_for(D);
            bool hit[CPL];
            bool any = false;
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                hit[s] = cid[s] != 0xffffffffu && exact_member<D>(qd, y[s], a.E2);
                any |= hit[s];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const uint32_t qid = (uint32_t)__double_as_longlong(qd[D]);
            const uint32_t ql = ql_base + qi;
            if (st.fill + 2 * 32 * CPL > (uint32_t)a.eb) flush(st, ws, a, lane);
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                bool self = false;
                if (home_chunk) {
                    const uint32_t k = kb + lane + 32 * s;
                    if (k < home_len) {
                        if (k < ql) hit[s] = false;
                        self = (k == ql);
                    }
                }
                const uint32_t np = hit[s] ? ((UNI && !self) ? 2u : 1u) : 0u;
                emit_slot(st, ws, a, lane, qid, cid[s], np);
            }
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- the kernel

// One join's pipelined loop for this warp: takes work items of the join
// until none is left, then flushes its staged pairs and adds its counters.
// The warp's mbarriers are initialised on entry and invalidated on a normal
// exit, so a warp can run several joins one after another in the same
// shared-memory area.  Returns false when a bounded wait expired.
template <int D, bool F32, bool UNI, int FR>
__device__ __forceinline__ bool join_body(const JoinArgs &a, const uint32_t *counts,
                                          unsigned char *smem, int warp, int lane) {
    constexpr int CPL = cpl_for(D, F32);
    constexpr int CB = 32 * CPL;
    const uint32_t nbuf = (uint32_t)a.nbuf;   // chunk ring depth (launch parameter)
    const uint32_t smask = a.slots > 1 ? 1u : 0u;   // item slot of a sequence number
    typedef typename std::conditional<F32, float, double>::type T;
    const WarpSmem ws = carve(smem, a, warp, nbuf);
    // record and chunk sizes are compile-time (the host checks the stride)
    const uint32_t rsb = (uint32_t)(rs_for(D, F32) * sizeof(T));
    constexpr int sm_chunk = (CB * rs_for(D, F32) * (int)sizeof(T) + 15) & ~15;
    const unsigned char *rec = F32 ? reinterpret_cast<const unsigned char *>(a.rec32)
                                   : reinterpret_cast<const unsigned char *>(a.rec64);

    if (lane == 0)
        for (uint32_t i = 0; i < nbuf; ++i) mbar_init(&ws.bar[i], 1);
    fence_proxy_async_smem();
    __syncwarp();

    // counts[0] = |G|, counts[1] = number of work items (device-side, so the
    // launch needs no read-back)
    const uint32_t n_cells = *a.ccells;   // non-empty candidate cells (binary search of B)
    uint32_t item_end = a.item_end;
    if (counts[1] < item_end) item_end = counts[1];

    Pipe st;
    st.grab_pos = st.grab_end = 0;
    st.issued = st.consumed = 0;
    st.p_slot = st.c_slot = st.c_phase = 0;
    st.prod_seq = st.cons_seq = 0;
    st.p_chunk = st.c_chunk = 0;
    st.rcur = 0;
    st.fill = 0;
    st.prod_done = false;
    unsigned long long evals = 0, rechecks = 0;
    bool failed = false;

    uint2 it;
    // the first item with at least one candidate (in a two-set join a query
    // cell may have no candidate point around it: nothing to compare)
    bool have = false;
    while (!have && fetch_item(st, a, item_end, lane, it)) {
        prepare_item<D, F32, UNI>(ws, 0, it, a, n_cells, lane, evals);
        have = ws.hdr[0].nchunks != 0;
    }
    if (have) {
        for (;;) {
            // producer: keep up to nbuf chunks in flight, crossing into the
            // next item (at most one item ahead of the consumer)
            while (st.issued - st.consumed < nbuf) {
                const int ps = st.prod_seq & smask;
                if (st.p_chunk == ws.hdr[ps].nchunks) {
                    // a slot is free once the consumer has left its item:
                    // with two slots the producer runs one item ahead,
                    // with one it waits for the consumer to finish
                    if (st.prod_done || st.prod_seq + 1 >= st.cons_seq + (uint32_t)a.slots) break;
                    if (!fetch_item(st, a, item_end, lane, it)) {
                        st.prod_done = true;
                        break;
                    }
                    const int ns = (st.prod_seq + 1) & smask;
                    prepare_item<D, F32, UNI>(ws, ns, it, a, n_cells, lane, evals);
                    // an item without candidates is done: the next one may
                    // take the same slot
                    if (ws.hdr[ns].nchunks == 0) continue;
                    ++st.prod_seq;
                    st.p_chunk = 0;
                    st.rcur = 0;
                    continue;
                }
                // test hook: one warp never issues its first chunk, so its
                // wait for that chunk runs out (no copy is in flight for it)
                if (!(a.stall && st.issued == 0 && blockIdx.x == 0 && warp == 0))
                    issue_chunk<CB>(ws, ps, st.p_chunk, (int)st.p_slot, st.rcur, rec, rsb, lane,
                                    sm_chunk);
                ++st.issued;
                ++st.p_chunk;
                st.p_slot = st.p_slot + 1 == nbuf ? 0u : st.p_slot + 1;
            }
            if (st.consumed == st.issued) break;
            // consumer
            const int r = (int)st.c_slot;
            if (!mbar_wait_bounded(&ws.bar[r], st.c_phase, a.timeout_ns)) {
                failed = true;
                if (lane == 0) atomicOr(a.error, kErrTimeout);
                // let the other copies in flight land before leaving
                for (uint32_t k = st.consumed + 1; k < st.issued; ++k)
                    (void)mbar_wait_bounded(&ws.bar[k % nbuf], (k / nbuf) & 1u, a.timeout_ns);
                break;
            }
            consume_chunk<D, F32, UNI, FR>(st, ws, st.cons_seq & smask, st.c_chunk, r, a, lane,
                                           rechecks);
            ++st.consumed;
            ++st.c_chunk;
            if (++st.c_slot == nbuf) {
                st.c_slot = 0;
                st.c_phase ^= 1u;
            }
            if (st.c_chunk == ws.hdr[st.cons_seq & smask].nchunks) {
                ++st.cons_seq;
                st.c_chunk = 0;
            }
        }
    }
    if (!failed) flush(st, ws, a, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
    if (lane == 0) {
        if (evals) atomicAdd(&a.counter[1], evals);
        if (rechecks) atomicAdd(&a.counter[2], rechecks);
        // every copy issued has been waited for: the barriers are idle
        if (!failed)
            for (uint32_t i = 0; i < nbuf; ++i) mbar_inval(&ws.bar[i]);
    }
    __syncwarp();
    return !failed;
}

template <int D, bool F32, bool UNI, int FR>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, minb_for(D, F32))
    join_kernel(const JoinArgs a, const uint32_t *counts) {
    extern __shared__ __align__(128) unsigned char smem[];
    (void)join_body<D, F32, UNI, FR>(a, counts, smem, threadIdx.x >> 5, threadIdx.x & 31);
}

// Many joins in one persistent launch: every warp takes part in the joins in
// the order given, moving on to the next join as soon as the current one
// has no work item left for it (no barrier between joins, so the tail of one
// join overlaps the start of the next).  Each join has its own work cursor,
// counters, output and error word; its dimension and precision select the
// specialised loop.  The job table lives in the kernel parameters (constant
// bank), read with warp-uniform indices.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2)
    multi_join_kernel(const __grid_constant__ MultiJobs m) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (uint32_t j = 0; j < m.n; ++j) {
        const JoinArgs &a = m.job[j];
        bool ok = true;
        switch (a.d * 2 + (a.f32 ? 1 : 0)) {
#define SJ_MJ_CASE(DD)                                                                  \
    case 2 * DD: ok = join_body<DD, false, true, 0>(a, a.dcounts, smem, warp, lane); break; \
    case 2 * DD + 1: ok = join_body<DD, true, true, 2>(a, a.dcounts, smem, warp, lane); break;
            SJ_MJ_CASE(1)
            SJ_MJ_CASE(2)
            SJ_MJ_CASE(3)
            SJ_MJ_CASE(4)
            SJ_MJ_CASE(5)
            SJ_MJ_CASE(6)
            SJ_MJ_CASE(7)
            SJ_MJ_CASE(8)
#undef SJ_MJ_CASE
            default: break;
        }
        if (!ok) return;
    }
}

typedef JoinKernelFn KernelFn;

// The FP32 kernels come in a grid-frame and a cell-frame variant, so that
// each inlines one candidate transform only.
template <int D>
KernelFn pick(bool f32, bool uni, bool cell) {
    if (f32 && cell) return uni ? join_kernel<D, true, true, 1> : join_kernel<D, true, false, 1>;
    if (f32) return uni ? join_kernel<D, true, true, 0> : join_kernel<D, true, false, 0>;
    return uni ? join_kernel<D, false, true, 0> : join_kernel<D, false, false, 0>;
}

KernelFn pick_kernel(int d, bool f32, bool uni, bool cell) {
    switch (d) {
        case 1: return pick<1>(f32, uni, cell);
        case 2: return pick<2>(f32, uni, cell);
        case 3: return pick<3>(f32, uni, cell);
        case 4: return pick<4>(f32, uni, cell);
        case 5: return pick<5>(f32, uni, cell);
        case 6: return pick<6>(f32, uni, cell);
        case 7: return pick<7>(f32, uni, cell);
        case 8: return pick<8>(f32, uni, cell);
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

sj_status block_shape_uncached(Error &err, const void *fn, int sm_warp, int force_wpb, int dev,
                               int *wpb_out, int *per_sm_out);

// Warps per block of a join launch: the block size (8, 4, 2 or 1 warps)
// that keeps the most warps resident per SM under the shared-memory and
// register limits, or force_wpb when given and it fits.
sj_status block_shape(Error &err, const void *fn, int sm_warp, int force_wpb, int dev, int *wpb_out,
                      int *per_sm_out) {
    // answers are cached: the occupancy queries cost more host time than a
    // small join kernel takes on the device
    static std::mutex cache_mu;
    static std::map<std::tuple<const void *, int, int, int>, std::pair<int, int>> cache;
    const auto key = std::make_tuple(fn, sm_warp, force_wpb, dev);
    {
        std::lock_guard<std::mutex> lk(cache_mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *wpb_out = it->second.first;
            *per_sm_out = it->second.second;
            return SJ_OK;
        }
    }
    const sj_status st = block_shape_uncached(err, fn, sm_warp, force_wpb, dev, wpb_out, per_sm_out);
    if (st == SJ_OK) {
        std::lock_guard<std::mutex> lk(cache_mu);
        cache[key] = std::make_pair(*wpb_out, *per_sm_out);
    }
    return st;
}

sj_status block_shape_uncached(Error &err, const void *fn, int sm_warp, int force_wpb, int dev,
                               int *wpb_out, int *per_sm_out) {
    int smem_optin = 0;
    SJ_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    {
        // the limit is only ever raised, so that a launch prepared by another
        // thread never finds it lowered under its shared-memory size
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        cudaFuncAttributes fa;
        SJ_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
        const int want = std::min(smem_optin, sm_warp * kWarpsPerBlock);
        if (fa.maxDynamicSharedSizeBytes < want)
            SJ_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, want));
    }
    for (int pass = 0; pass < 2; ++pass) {
        int wpb = 0, per_sm = 0, best = 0;
        for (int w = kWarpsPerBlock; w >= 1; w /= 2) {
            if (pass == 0 && force_wpb > 0 && w != force_wpb) continue;
            if ((size_t)sm_warp * w > (size_t)smem_optin) continue;
            int b = 0;
            SJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, w * 32, (size_t)sm_warp * w));
            if (b * w > best) { best = b * w; wpb = w; per_sm = b; }
        }
        if (best > 0) {
            *wpb_out = wpb;
            *per_sm_out = per_sm;
            return SJ_OK;
        }
        if (force_wpb <= 0) break;
    }
    return fail(err, SJ_EINVAL, "join kernel does not fit on an SM");
}

const void *multi_join_fn() { return reinterpret_cast<const void *>(multi_join_kernel); }

namespace {

// Entry t of the template table of (d, UNICOMP) (format in join_dev.cuh).
uint32_t template_entry(int d, bool uni, uint32_t t) {
    uint32_t pow3[kMaxDim + 1];
    pow3[0] = 1;
    for (int j = 1; j <= kMaxDim; ++j) pow3[j] = 3 * pow3[j - 1];
    int dy[kMaxDim] = {0};
    uint32_t xm = 3, gate = 8;
    if (uni) {
        if (t == 0) {
            xm = 0;
        } else if (t <= 2) {
            xm = t;            // 1: x - 1, 2: x + 1
            gate = 0;
        } else {
            const uint32_t u = t - 3;
            int k = 1;
            for (int kk = 1; kk < d; ++kk)
                if (u >= pow3[kk] - 1) k = kk + 1;
            gate = (uint32_t)k;
            const uint32_t p = pow3[k - 1];
            const uint32_t v = u - (p - 1);
            uint32_t rem = v % p;
            for (int j = 1; j < k; ++j) {
                dy[j] = (int)(rem % 3) - 1;
                rem /= 3;
            }
            dy[k] = (v / p) ? 1 : -1;
        }
    } else {
        uint32_t rem = t;
        for (int j = 1; j < d; ++j) {
            dy[j] = (int)(rem % 3) - 1;
            rem /= 3;
        }
    }
    uint32_t e = xm | (gate << 2);
    for (int j = 1; j < d; ++j) e |= (uint32_t)(dy[j] + 1) << (6 + 2 * (j - 1));
    return e;
}

uint32_t template_offset(int d, bool uni) {
    uint32_t off = 0;
    for (int dd = 1; dd <= kMaxDim; ++dd)
        for (int u = 0; u < 2; ++u) {
            if (dd == d && (u == 1) == uni) return off;
            off += (uint32_t)n_templates(dd, u == 1);
        }
    return off;
}

std::mutex g_tmpl_mu;
const uint32_t *g_tmpl_dev[64] = {nullptr};

// Device address of the template table of (d, UNICOMP) on the current
// device; the tables are written on the first use on each device.
sj_status template_table(Error &err, int d, bool uni, const uint32_t **out) {
    int dev = 0;
    SJ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(err, SJ_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_tmpl_mu);
    if (!g_tmpl_dev[dev]) {
        std::vector<uint32_t> h;
        h.reserve(kTemplateEntries);
        for (int dd = 1; dd <= kMaxDim; ++dd)
            for (int u = 0; u < 2; ++u)
                for (int t = 0; t < n_templates(dd, u == 1); ++t) h.push_back(template_entry(dd, u == 1, t));
        if (h.size() != (size_t)kTemplateEntries) return fail(err, SJ_ECUDA, "template table size");
        SJ_CUDA_TRY(cudaMemcpyToSymbol(g_templates, h.data(), h.size() * sizeof(uint32_t)));
        void *p = nullptr;
        SJ_CUDA_TRY(cudaGetSymbolAddress(&p, g_templates));
        g_tmpl_dev[dev] = static_cast<const uint32_t *>(p);
    }
    *out = g_tmpl_dev[dev] + template_offset(d, uni);
    return SJ_OK;
}

}  // namespace

sj_status fill_join_args(Error &err, const Index &ix, const JoinLaunch &cfg, uint32_t item_begin,
                         uint32_t item_end, uint2 *out, uint64_t cap,
                         unsigned long long *d_counter, uint32_t *d_work, uint32_t *d_error,
                         int count_only, JoinArgs &a, const Index *qix) {
    const Geometry &g = ix.g;
    const int d = g.d;
    const bool f32 = cfg.prec_fp32 && g.fp32_ok;
    const bool uni = cfg.unicomp != 0;
    const bool hd = ix.dfull > kMaxDim;
    if (!f32 && !(hd ? ix.recd64.p : ix.rec64.p)) return fail(err, SJ_EINVAL, "FP64 records missing");
    if (hd && qix) return fail(err, SJ_EINVAL, "two-set joins take at most 8 dimensions");
    // the query side (work items, home cells, query points): another index
    // on the same grid for a two-set join, else the candidate index itself
    const Index &q = qix ? *qix : ix;
    if (qix && (uni || !(f32 || q.rec64.p)))
        return fail(err, SJ_EINVAL, "two-set joins search all adjacent cells and need both records");
    if (qix && f32 && (q.g.frame != g.frame || !q.g.fp32_ok))
        return fail(err, SJ_EINVAL, "two-set join indexes with different FP32 frames");
    memset(&a, 0, sizeof(a));
    a.qrec32 = static_cast<const float *>(q.rec32.p);
    a.qrec64 = static_cast<const double *>(q.rec64.p);
    a.qpts = static_cast<const double *>(q.pts.p);
    a.qG = static_cast<const uint32_t *>(q.G.p);
    a.qcc = static_cast<const int32_t *>(q.cc.p);
    a.ccells = n_items_dev(ix) - 1;
    a.rec32 = static_cast<const float *>(ix.rec32.p);
    a.rec64 = static_cast<const double *>(ix.rec64.p);
    a.pts = static_cast<const double *>(ix.pts.p);
    a.G = static_cast<const uint32_t *>(ix.G.p);
    a.B = static_cast<const uint64_t *>(ix.B.p);
    a.cc = static_cast<const int32_t *>(ix.cc.p);
    a.M = static_cast<const uint32_t *>(ix.M.p);
    a.lut = static_cast<const uint32_t *>(ix.lut.p);
    a.items = static_cast<const uint2 *>(q.items.p);
    a.item_begin = item_begin;
    a.item_end = item_end;
    a.item_stride = cfg.item_stride > 0 ? cfg.item_stride : 1;
    a.mwords = ix.mwords;
    a.dense = ix.dense;
    a.tuple = ix.tuple;
    a.rs = f32 ? ix.rs32 : ix.rs64;
    a.n_templates = n_templates(d, uni);
    SJ_TRY(template_table(err, d, uni, &a.tmpl));
    for (int j = 0; j < d; ++j) {
        a.ng[j] = (int32_t)g.ng[j];
        a.stride[j] = g.stride[j];
    }
    a.lo32 = g.lo32;
    a.hi32 = g.hi32;
    a.w32 = g.w32;
    a.w4 = g.w4;
    a.inv_w4 = g.inv_w4;
    a.frame = f32 ? g.frame : SJ_FRAME_GRID;
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
    // query record: FP32 m_0 .. m_{d-1}, pp, id -> d + 2 floats;
    // FP64: x_0..x_{d-1}, id
    a.qrs = f32 ? qrs32_for(d) : rs64_for(d);
    // the search kernel takes the record strides as compile-time constants
    if (!hd && a.rs != rs_for(d, f32)) return fail(err, SJ_EINVAL, "record stride");
    a.cb = 32 * cpl_for(d, f32);
    a.sm_ranges = round16(a.n_templates * (int)sizeof(uint2));
    a.sm_queries = round16(kQueryBlock * a.qrs * esz);
    a.sm_chunk = round16(a.cb * rsb);
    // staging area: the launch's choice (128 .. 1024 pairs) or by d
    a.eb = (cfg.eb == 128 || cfg.eb == 256 || cfg.eb == 512 || cfg.eb == 1024) ? cfg.eb : emit_for(d, f32);
    a.sm_emit = round16(a.eb * (int)sizeof(uint2));
    // ring depth: the launch's choice (2..8 chunks; the warp has 8 mbarriers)
    a.nbuf = (cfg.nbuf >= 2 && cfg.nbuf <= 8) ? cfg.nbuf : nbuf_for(d, f32);
    a.slots = (cfg.slots == 1 || cfg.slots == 2) ? cfg.slots : slots_for(d, f32);
    a.sm_warp = 64 + round16(a.slots * (int)sizeof(ItemHdr)) + a.slots * a.sm_ranges +
                a.slots * a.sm_queries + a.nbuf * a.sm_chunk + a.sm_emit;
    a.timeout_ns = cfg.timeout_ns > 0 ? cfg.timeout_ns : 2000000000ull;
    a.stall = cfg.stall;
    a.d = d;
    a.f32 = f32 ? 1 : 0;
    a.dcounts = n_items_dev(q) - 1;
    if (hd) {
        // the high-dimensional kernel: ranges, then the staged query records
        a.recd32 = static_cast<const float *>(ix.recd32.p);
        a.recd64 = static_cast<const double *>(ix.recd64.p);
        a.ptsd = static_cast<const double *>(ix.ptsd.p);
        a.dfull = ix.dfull;
        a.rsd = f32 ? ix.rsd32 : ix.rsd64;
        // staged query: 4 ceil(d / 4) value pairs (two floats or one double
        // each); the expanded form takes fewer (4 ceil(d / 4) + 4 floats)
        a.sm_queries = round16(kQueryBlock * 4 * ((ix.dfull + 3) / 4) * 8);
        // the expanded form's origin: 4 ceil(d / 4) floats per warp
        a.sm_warp = a.sm_ranges + a.sm_queries + 64;
        a.hd_exp = ix.hd_exp;
        a.hmid = static_cast<const float *>(ix.hmid_dev.p);
        a.hgrid4 = ~0ull;
        for (int t = 0; t < kHdGridDims && t < ix.g.d; ++t)
            a.hgrid4 &= ~(0xfull << (4 * ix.gdim[t])) | ((uint64_t)t << (4 * ix.gdim[t]));
    }
    return SJ_OK;
}

sj_status launch_join(Error &err, const Index &ix, const JoinLaunch &cfg, uint32_t item_begin,
                      uint32_t item_end, uint2 *out, uint64_t cap,
                      unsigned long long *d_counter, uint32_t *d_work, uint32_t *d_error,
                      int count_only, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                      const Index *qix) {
    JoinArgs a;
    SJ_TRY(fill_join_args(err, ix, cfg, item_begin, item_end, out, cap, d_counter, d_work, d_error,
                          count_only, a, qix));
    const int d = a.d;
    const bool f32 = a.f32 != 0;
    const bool uni = cfg.unicomp != 0;

    KernelFn fn = ix.dfull > kMaxDim ? hd_kernel_fn(ix.dfull, f32, uni, ix.hd_exp != 0)   // hd_join.cu
                                     : pick_kernel(d, f32, uni, a.frame == SJ_FRAME_CELL);
    if (!fn) return fail(err, SJ_EINVAL, "unsupported dimension");
    int dev = 0;
    SJ_CUDA_TRY(cudaGetDevice(&dev));
    int wpb = 0, per_sm = 0;
    SJ_TRY(block_shape(err, reinterpret_cast<const void *>(fn), a.sm_warp, cfg.wpb, dev, &wpb, &per_sm));
    const size_t smem = (size_t)a.sm_warp * wpb;
    int blocks = cfg.blocks > 0 ? cfg.blocks : per_sm * sm_count(dev);
    if (item_end <= item_begin) blocks = 1;
    SJ_CUDA_TRY(cudaMemsetAsync(d_work, 0, sizeof(uint32_t), s));
    if (ev0) SJ_CUDA_TRY(cudaEventRecord(ev0, s));
    fn<<<blocks, wpb * 32, smem, s>>>(a, a.dcounts); note_launch();
    SJ_CUDA_TRY(cudaGetLastError());
    if (ev1) SJ_CUDA_TRY(cudaEventRecord(ev1, s));
    return SJ_OK;
}

}  // namespace sj
