// api.cu -- the C ABI of include/sj.h.
//
// Contexts own two streams (kernels, host copies), a stream-ordered device
// memory pool, small device counters and a pinned read-back area.  Host
// results live in pinned buffers drawn from a process-wide cache, so result
// batches are copied straight from device memory into the caller's result
// (Section V-A's overlapped transfers) and a repeated join reuses them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "engine.cuh"
#include "sj_internal.cuh"

namespace sj {

void set_cuda_error(Error &err, cudaError_t e, const char *expr, const char *file, int line) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "CUDA error %d (%s) at %s:%d in %s", (int)e,
                  cudaGetErrorString(e), file, line, expr);
    err.msg = buf;
    err.st = (e == cudaErrorMemoryAllocation) ? SJ_ENOMEM : SJ_ECUDA;
}

sj_status fail(Error &err, sj_status st, const std::string &msg) {
    err.st = st;
    err.msg = msg;
    return st;
}

sj_status dev_alloc(Error &err, DevBuf &b, size_t bytes, cudaStream_t s) {
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        std::snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", bytes,
                      cudaGetErrorString(e));
        return fail(err, e == cudaErrorMemoryAllocation ? SJ_ENOMEM : SJ_ECUDA, buf);
    }
    b.p = p;
    b.bytes = bytes;
    return SJ_OK;
}

void dev_free(DevBuf &b, cudaStream_t s) {
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.bytes = 0;
}

namespace {
std::atomic<uint64_t> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device < 0) cudaGetDevice(&device);
    if (device < 0 || device >= 64) return 1;
    if (!cached[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cached[device] = v > 0 ? v : 1;
    }
    return cached[device];
}

// ---------------------------------------------------------------- pinned cache

namespace {

struct PinnedCache {
    std::mutex mu;
    std::multimap<size_t, void *> free_list;
    size_t cached = 0;
    static constexpr size_t kLimit = (size_t)32 << 30;

    // Buffers are allocated in size classes (eight per power of two, at
    // least 64 KiB) so that a freed buffer serves later requests of about
    // the same size: pinning fresh memory costs far more than the slack.
    static size_t size_class(size_t bytes) {
        size_t c = (size_t)64 << 10;
        if (bytes <= c) return c;
        size_t p = 1;
        while (p <= bytes / 2) p <<= 1;      // largest power of two <= bytes
        const size_t step = p / 8;
        return (bytes + step - 1) / step * step;
    }
    void *get(size_t bytes, size_t *got) {
        bytes = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = free_list.lower_bound(bytes);
            if (it != free_list.end() && it->first <= bytes * 2 + ((size_t)64 << 20)) {
                void *p = it->second;
                *got = it->first;
                cached -= it->first;
                free_list.erase(it);
                return p;
            }
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        *got = bytes;
        return p;
    }
    void put(void *p, size_t bytes) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        if (cached + bytes > kLimit) {
            cudaFreeHost(p);
            return;
        }
        free_list.emplace(bytes, p);
        cached += bytes;
    }
};

PinnedCache &pinned_cache() {
    static PinnedCache *c = new PinnedCache();  // never destroyed: results may outlive contexts
    return *c;
}

}  // namespace

void *pinned_get(size_t bytes, size_t *got) { return pinned_cache().get(bytes, got); }
void pinned_put(void *p, size_t bytes) { pinned_cache().put(p, bytes); }

}  // namespace sj

namespace sj {

namespace {

// layout of ctx->misc (unsigned long long words)
constexpr int kMiscCounter = 0;   // [0..3] pairs, evaluations, rechecks, spare
constexpr int kMiscWork = 4;      // u32 cursor
constexpr int kMiscError = 5;     // u32 error word
constexpr int kMiscWords = 8;
constexpr int kEarlyCountsWord = 32;   // h_misc words of the early build counters

struct Scoped {
    sj_ctx *ctx;
    Error err;
    uint64_t launches0;
    explicit Scoped(sj_ctx *c) : ctx(c), launches0(launches_so_far()) {}
    sj_status done(sj_status st) {
        if (ctx) {
            ctx->last_err = (st == SJ_OK || st == SJ_PENDING) ? std::string() : err.msg;
            ctx->stats.kernel_launches = launches_so_far() - launches0;
        }
        return st;
    }
};

sj_status check_args(Error &err, const double *pts, uint64_t n, int d, double eps) {
    if (!pts) return fail(err, SJ_EINVAL, "pts is NULL");
    if (n == 0) return fail(err, SJ_EINVAL, "n must be positive");
    if (d < 1 || d > kMaxPointDim) return fail(err, SJ_EINVAL, "d must be in [1, 16]");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(err, SJ_EINVAL, "eps must be positive and finite");
    if (n >= (1ull << 32)) return fail(err, SJ_ERANGE, "n must be below 2^32");
    return SJ_OK;
}

sj_status set_device(Error &err, int dev) {
    SJ_CUDA_TRY(cudaSetDevice(dev));
    return SJ_OK;
}

unsigned long long *misc_dev(sj_ctx *ctx) { return static_cast<unsigned long long *>(ctx->misc.p); }

sj_status profile_events(Error &err, sj_ctx *ctx, cudaEvent_t *e0, cudaEvent_t *e1) {
    *e0 = *e1 = nullptr;
    if (!ctx->cfg.profile) return SJ_OK;
    if (ctx->prof_used == ctx->prof.size()) {
        cudaEvent_t a, b;
        SJ_CUDA_TRY(cudaEventCreate(&a));
        SJ_CUDA_TRY(cudaEventCreate(&b));
        ctx->prof.emplace_back(a, b);
    }
    *e0 = ctx->prof[ctx->prof_used].first;
    *e1 = ctx->prof[ctx->prof_used].second;
    ctx->prof_used++;
    return SJ_OK;
}

JoinLaunch default_launch(const sj_ctx *ctx) {
    JoinLaunch l;
    l.prec_fp32 = ctx->cfg.prec == SJ_PREC_FP32_RECHECK;
    l.unicomp = ctx->cfg.unicomp;
    l.grab = ctx->cfg.grab > 0 ? ctx->cfg.grab : 1;
    l.nbuf = ctx->cfg.nbuf > 0 ? ctx->cfg.nbuf : 0;
    l.eb = ctx->cfg.staging > 0 ? ctx->cfg.staging : 0;
    l.wpb = ctx->cfg.wpb > 0 ? ctx->cfg.wpb : 0;
    l.slots = ctx->cfg.slots > 0 ? ctx->cfg.slots : 0;
    l.timeout_ns = ctx->cfg.wait_ms > 0 ? (uint64_t)ctx->cfg.wait_ms * 1000000ull : 0;
    l.stall = ctx->cfg.test_stall ? 1 : 0;
    return l;
}

JoinLaunch launch_cfg(const sj_ctx *ctx) { return ctx->launch; }

// Launch parameters of the join on ix: the defaults, or with autotune = 1
// (and no launch parameter forced in the configuration) the tuner's choice for the
// index's key (|G| read on the host first, from the mid-build copy when there is one).
sj_status prepare_launch(Error &err, sj_ctx *ctx, Index &ix, cudaStream_t s) {
    ctx->launch = default_launch(ctx);
    ctx->launch_tuned = 0;
    // the tuned parameters belong to the main kernel, not the one for more
    // than 8 dimensions
    if (!ctx->cfg.autotune || launch_forced(ctx->cfg) || ix.dfull > kMaxDim) return SJ_OK;
    if (!ix.counts_read && ix.early_ev) {
        // |G| was copied mid-build: wait for that copy only, not the build
        SJ_CUDA_TRY(cudaEventSynchronize(ix.early_ev));
        ix.n_cells = ix.early_counts[1];
    } else {
        SJ_TRY(read_counts(err, ix, s));
    }
    return tune_launch(err, ix, ctx->launch, s, &ctx->launch_tuned);
}

// Build options of a call whose index lives only inside the call: device
// points are read in place and |G| is copied to the host mid-build.
BuildOpts call_build_opts(sj_ctx *ctx) {
    BuildOpts o;
    o.borrow_pts = true;
    if (ctx->ev_counts) {
        o.h_counts = reinterpret_cast<uint32_t *>(ctx->h_misc + kEarlyCountsWord);
        o.ev_counts = ctx->ev_counts;
    }
    return o;
}

void record_launch(sj_ctx *ctx, const Index &ix) {
    ctx->stats.frame = (ctx->cfg.prec == SJ_PREC_FP32_RECHECK && ix.g.fp32_ok) ? ix.g.frame : -1;
    ctx->stats.grab = ctx->launch.grab;
    ctx->stats.nbuf = ctx->launch.nbuf;
    ctx->stats.wpb = ctx->launch.wpb;
    ctx->stats.staging = ctx->launch.eb;
    ctx->stats.tuned = ctx->launch_tuned;
}

// Runs one join launch over items [ib, ie) into out (cap pairs) and reads
// the counters back.  Synchronises stream s.
sj_status join_once(Error &err, sj_ctx *ctx, const Index &ix, uint32_t ib, uint32_t ie,
                    uint32_t stride, uint2 *out, uint64_t cap, int count_only, cudaStream_t s,
                    unsigned long long res[3]) {
    unsigned long long *m = misc_dev(ctx);
    SJ_CUDA_TRY(cudaMemsetAsync(m, 0, kMiscWords * sizeof(unsigned long long), s));
    cudaEvent_t e0, e1;
    SJ_TRY(profile_events(err, ctx, &e0, &e1));
    JoinLaunch l = launch_cfg(ctx);
    l.item_stride = stride;
    SJ_TRY(launch_join(err, ix, l, ib, ie, out, cap, m + kMiscCounter,
                       reinterpret_cast<uint32_t *>(m + kMiscWork),
                       reinterpret_cast<uint32_t *>(m + kMiscError), count_only, s, e0, e1));
    SJ_CUDA_TRY(cudaMemcpyAsync(ctx->h_misc, m, kMiscWords * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, s));
    SJ_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t errw = (uint32_t)ctx->h_misc[kMiscError];
    if (errw & kErrTimeout) return fail(err, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
    res[0] = ctx->h_misc[0];
    res[1] = ctx->h_misc[1];
    res[2] = ctx->h_misc[2];
    return SJ_OK;
}

// Sampled work items of the first pair-count estimate (one segment), and of
// the estimate by segments that follows when the result needs more than
// the minimum number of batches.  A sampled launch is latency-bound (a few
// items per warp), so its time grows slowly with the sample.
constexpr uint32_t kEstimateSamples = 4096;
constexpr uint32_t kSegmentSamples = 16384;

// Pair-count estimates of S equal segments of the work items, each from a
// systematic sample (every stride-th item, about `samples` sampled items in
// all): the S count-only launches run back to back on s, each into its
// own counters, with one read-back at the end.  Pair density varies along
// the cell order (cells at the boundary of the data have fewer
// neighbours), so the batches are later cut at equal estimated pairs, not
// at equal item counts.
sj_status estimate_segments(Error &err, sj_ctx *ctx, const Index &ix, cudaStream_t s, uint32_t S,
                            uint32_t samples, std::vector<double> &seg) {
    const uint32_t ni = ix.n_items;
    const uint32_t stride = ni > samples ? ni / samples : 1;
    seg.assign(S, 0.0);
    DevBuf ctr;
    SJ_TRY(dev_alloc(err, ctr, (size_t)S * 4 * sizeof(unsigned long long), s));
    unsigned long long *c = static_cast<unsigned long long *>(ctr.p);
    unsigned long long *m = misc_dev(ctx);
    auto run = [&]() -> sj_status {
        SJ_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)S * 4 * sizeof(unsigned long long), s));
        SJ_CUDA_TRY(cudaMemsetAsync(m, 0, kMiscWords * sizeof(unsigned long long), s));
        JoinLaunch l = launch_cfg(ctx);
        l.item_stride = stride;
        for (uint32_t q = 0; q < S; ++q) {
            const uint32_t lo = (uint32_t)((uint64_t)ni * q / S), hi = (uint32_t)((uint64_t)ni * (q + 1) / S);
            if (hi <= lo) continue;
            SJ_TRY(launch_join(err, ix, l, lo, hi, nullptr, 0, c + 4 * q,
                               reinterpret_cast<uint32_t *>(m + kMiscWork),
                               reinterpret_cast<uint32_t *>(m + kMiscError), 1, s, nullptr, nullptr));
        }
        std::vector<unsigned long long> h((size_t)S * 4);
        SJ_CUDA_TRY(cudaMemcpyAsync(h.data(), c, h.size() * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaMemcpyAsync(ctx->h_misc, m, kMiscWords * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        if ((uint32_t)ctx->h_misc[kMiscError] & kErrTimeout)
            return fail(err, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
        for (uint32_t q = 0; q < S; ++q) {
            const uint32_t lo = (uint32_t)((uint64_t)ni * q / S), hi = (uint32_t)((uint64_t)ni * (q + 1) / S);
            if (hi <= lo) continue;
            const uint64_t sampled = (hi - lo + stride - 1) / stride;
            seg[q] = (double)h[4 * q] * (double)(hi - lo) / (double)sampled;
        }
        return SJ_OK;
    };
    const sj_status st = run();
    dev_free(ctr, s);
    return st;
}

// Where the batches of a host-output join go.
struct HostSink {
    sj_result *res = nullptr;        // gather mode
    sj_chunk_cb cb = nullptr;        // callback mode
    void *user = nullptr;
    bool stop = false;
};

sj_status grow_result(Error &err, sj_result *r, uint64_t need_pairs) {
    const size_t need = (size_t)need_pairs * 8;
    if (need <= r->bytes && r->pairs) return SJ_OK;
    size_t want = std::max(need, r->bytes + r->bytes / 2);
    want = (want + 4095) & ~(size_t)4095;
    size_t got = 0;
    void *p = pinned_cache().get(want, &got);
    if (!p) return fail(err, SJ_ENOMEM, "pinned host allocation failed");
    if (r->pairs) {
        std::memcpy(p, r->pairs, (size_t)r->count * 8);
        pinned_cache().put(r->pairs, r->bytes);
    }
    r->pairs = static_cast<uint32_t *>(p);
    r->bytes = got;
    return SJ_OK;
}

// Result batching (Section V-A): the work items are split into contiguous
// ranges; batch b's kernel writes into device buffer b % 2 while batch
// b-1's pairs are copied to the host on the copy stream.
sj_status run_batches(Error &err, sj_ctx *ctx, Index &ix, HostSink &sink) {
    cudaStream_t s = ctx->s_main, sc = ctx->s_copy;
    SJ_TRY(read_counts(err, ix, s));
    const uint32_t ni = ix.n_items;
    const uint64_t cap_total = ctx->cfg.out_cap_bytes ? ctx->cfg.out_cap_bytes : (2ull << 30);
    const uint64_t bufcap_max = std::max<uint64_t>(cap_total / 16, 4096);  // pairs per buffer
    const uint64_t min_nb = (uint64_t)std::max(1, ctx->cfg.min_batches);
    auto batches_for = [&](uint64_t e) {
        const uint64_t padded = e + e / 8 + 4096;
        uint64_t b = std::max<uint64_t>((padded + bufcap_max - 1) / bufcap_max, min_nb);
        return std::min<uint64_t>(b, ni ? ni : 1);
    };
    // one sampled estimate; when the result needs more than the minimum
    // number of batches, a second one by segments (enough to follow the
    // density along the cell order, each still sampling about 256 items or
    // more) to cut the batches at equal estimated pairs
    std::vector<double> seg;
    SJ_TRY(estimate_segments(err, ctx, ix, s, 1, kEstimateSamples, seg));
    uint32_t S = 1;
    if (batches_for((uint64_t)seg[0]) > min_nb) {
        S = std::max<uint32_t>(1, std::min<uint32_t>(64, ni / 4096));
        if (S > 1) SJ_TRY(estimate_segments(err, ctx, ix, s, S, kSegmentSamples, seg));
    }
    double est_d = 0;
    for (double v : seg) est_d += v;
    const uint64_t est = (uint64_t)est_d;
    ctx->stats.estimate = est;
    const uint64_t padded = est + est / 8 + 4096;
    const uint64_t nb_eq = batches_for(est);
    uint64_t bufcap = std::min<uint64_t>(bufcap_max, padded / nb_eq + padded / (4 * nb_eq) + 65536);
    // Batch 0's kernel overlaps no copy, and the last batch's copy overlaps
    // no kernel, while every other batch's kernel overlaps the copy of the
    // one before: a small first and a small last batch (1/16 of the
    // estimated pairs each, or less) leave little of the join or of the
    // copies exposed, and the rest is cut into nb_eq batches of equal
    // estimated pairs.  Batch b covers items [cut[b], cut[b+1]); the
    // cumulative estimate is interpolated linearly inside a segment.
    const bool edges = nb_eq >= 2 && ni >= 2 * nb_eq + 4;
    const uint64_t nb = nb_eq + (edges ? 2 : 0);
    const double f0 = edges ? std::min(1.0 / 16.0, 0.5 / (double)nb_eq) : 0.0;
    std::vector<uint32_t> cut(nb + 1, 0);
    cut[nb] = ni;
    {
        double acc = 0;
        uint32_t q = 0;
        for (uint64_t b = 1; b < nb; ++b) {
            const double frac = edges ? f0 + (1.0 - 2.0 * f0) * (double)(b - 1) / (double)nb_eq
                                      : (double)b / (double)nb;
            const double target = est_d * frac;
            while (q < S && acc + seg[q] < target) acc += seg[q++];
            uint32_t x;
            if (q >= S) {
                x = ni;
            } else {
                const double lo = (double)ni * q / S, hi = (double)ni * (q + 1) / S;
                const double f = seg[q] > 0 ? (target - acc) / seg[q] : 0.0;
                x = (uint32_t)std::min<double>(hi, lo + f * (hi - lo));
            }
            cut[b] = std::max(cut[b - 1], std::min(x, ni));
        }
    }

    DevBuf dbuf[2];
    SJ_TRY(dev_alloc(err, dbuf[0], bufcap * 8, s));
    sj_status st = dev_alloc(err, dbuf[1], bufcap * 8, s);
    if (st != SJ_OK) { dev_free(dbuf[0], s); return st; }
    DevBuf ctr;
    st = dev_alloc(err, ctr, nb * 4 * sizeof(unsigned long long) + 64, s);
    if (st != SJ_OK) { dev_free(dbuf[0], s); dev_free(dbuf[1], s); return st; }
    unsigned long long *d_ctr = static_cast<unsigned long long *>(ctr.p);
    unsigned long long *h_ctr = nullptr;
    size_t h_ctr_bytes = 0;
    h_ctr = static_cast<unsigned long long *>(pinned_cache().get(nb * 4 * 8 + 64, &h_ctr_bytes));
    void *stage[2] = {nullptr, nullptr};
    size_t stage_bytes[2] = {0, 0};
    std::vector<cudaEvent_t> ev;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(sc);
        dev_free(dbuf[0], s);
        dev_free(dbuf[1], s);
        dev_free(ctr, s);
        if (h_ctr) pinned_cache().put(h_ctr, h_ctr_bytes);
        for (int i = 0; i < 2; ++i)
            if (stage[i]) pinned_cache().put(stage[i], stage_bytes[i]);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    };
#define SJ_R(expr) do { st = (expr); if (st != SJ_OK) { cleanup(); return st; } } while (0)
#define SJ_RC(expr) do { cudaError_t e__ = (expr); if (e__ != cudaSuccess) { set_cuda_error(err, e__, #expr, __FILE__, __LINE__); cleanup(); return err.st; } } while (0)
    if (!h_ctr) { cleanup(); return fail(err, SJ_ENOMEM, "pinned host allocation failed"); }
    if (sink.cb) {
        for (int i = 0; i < 2; ++i) {
            stage[i] = pinned_cache().get(bufcap * 8, &stage_bytes[i]);
            if (!stage[i]) { cleanup(); return fail(err, SJ_ENOMEM, "pinned host allocation failed"); }
        }
    } else {
        SJ_R(grow_result(err, sink.res, padded + padded / 8));
    }
    // events: kernel done (per batch), copy done (per buffer)
    ev.resize(nb + 2);
    for (auto &e : ev) SJ_RC(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t *ev_k = ev.data(), *ev_c = ev.data() + nb;

    std::vector<std::pair<uint32_t, uint32_t>> retry;
    std::vector<uint64_t> cb_pending;   // batch whose staged pairs await the callback
    uint64_t cb_count[2] = {0, 0};
    auto item_lo = [&](uint64_t b) { return cut[b]; };
    uint64_t batches_done = 0;

    auto launch_batch = [&](uint64_t b) -> sj_status {
        const int k = (int)(b & 1);
        if (b >= 2) SJ_CUDA_TRY(cudaStreamWaitEvent(s, ev_c[k], 0));
        unsigned long long *c = d_ctr + 4 * b;
        SJ_CUDA_TRY(cudaMemsetAsync(c, 0, 4 * sizeof(unsigned long long), s));
        cudaEvent_t e0, e1;
        SJ_TRY(profile_events(err, ctx, &e0, &e1));
        JoinLaunch l = launch_cfg(ctx);
        unsigned long long *m = misc_dev(ctx);
        SJ_TRY(launch_join(err, ix, l, item_lo(b), item_lo(b + 1), static_cast<uint2 *>(dbuf[k].p),
                           bufcap, c, reinterpret_cast<uint32_t *>(m + kMiscWork),
                           reinterpret_cast<uint32_t *>(m + kMiscError), 0, s, e0, e1));
        SJ_CUDA_TRY(cudaMemcpyAsync(h_ctr + 4 * b, c, 4 * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaEventRecord(ev_k[b], s));
        return SJ_OK;
    };
    auto deliver_cb = [&](int k) -> sj_status {
        // staged pairs of buffer k are complete once its copy event fired
        SJ_CUDA_TRY(cudaEventSynchronize(ev_c[k]));
        if (!sink.stop && cb_count[k])
            if (sink.cb(static_cast<const uint32_t *>(stage[k]), cb_count[k], sink.user) != 0)
                sink.stop = true;
        cb_count[k] = 0;
        return SJ_OK;
    };
    auto finish_batch = [&](uint64_t b) -> sj_status {
        const int k = (int)(b & 1);
        SJ_CUDA_TRY(cudaEventSynchronize(ev_k[b]));
        const uint64_t cnt = h_ctr[4 * b];
        ctx->stats.evaluations += h_ctr[4 * b + 1];
        ctx->stats.rechecks += h_ctr[4 * b + 2];
        batches_done++;
        if (cnt > bufcap) {
            retry.emplace_back(item_lo(b), item_lo(b + 1));
            SJ_CUDA_TRY(cudaEventRecord(ev_c[k], sc));
            return SJ_OK;
        }
        SJ_CUDA_TRY(cudaStreamWaitEvent(sc, ev_k[b], 0));
        ctx->stats.pairs += cnt;
        if (sink.cb) {
            if (cb_count[k]) SJ_TRY(deliver_cb(k));
            SJ_CUDA_TRY(cudaMemcpyAsync(stage[k], dbuf[k].p, cnt * 8, cudaMemcpyDeviceToHost, sc));
            cb_count[k] = cnt;
        } else {
            sj_result *r = sink.res;
            if ((r->count + cnt) * 8 > r->bytes) {
                SJ_CUDA_TRY(cudaStreamSynchronize(sc));
                SJ_TRY(grow_result(err, r, r->count + cnt));
            }
            SJ_CUDA_TRY(cudaMemcpyAsync(r->pairs + 2 * r->count, dbuf[k].p, cnt * 8,
                                        cudaMemcpyDeviceToHost, sc));
            r->count += cnt;
        }
        SJ_CUDA_TRY(cudaEventRecord(ev_c[k], sc));
        return SJ_OK;
    };

    for (uint64_t b = 0; b < nb; ++b) {
        if (sink.stop) break;
        SJ_R(launch_batch(b));
        if (b >= 1) SJ_R(finish_batch(b - 1));
    }
    if (!sink.stop) SJ_R(finish_batch(nb - 1));
    if (sink.cb) {
        for (int k = 0; k < 2; ++k) SJ_R(deliver_cb(k));
    }
    SJ_RC(cudaStreamSynchronize(sc));
    ctx->stats.batches = (uint32_t)batches_done;
    {
        unsigned long long *m = misc_dev(ctx);
        SJ_RC(cudaMemcpyAsync(ctx->h_misc, m, kMiscWords * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, s));
        SJ_RC(cudaStreamSynchronize(s));
        if ((uint32_t)ctx->h_misc[kMiscError] & kErrTimeout) {
            cleanup();
            return fail(err, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
        }
    }

    // overflowed batches: re-run in halves, synchronously
    while (!retry.empty() && !sink.stop) {
        std::pair<uint32_t, uint32_t> rg = retry.back();
        retry.pop_back();
        ctx->stats.retries++;
        unsigned long long r3[3];
        SJ_R(join_once(err, ctx, ix, rg.first, rg.second, 1, static_cast<uint2 *>(dbuf[0].p), bufcap,
                       0, s, r3));
        const uint64_t cnt = r3[0];
        if (cnt > bufcap) {
            if (rg.second - rg.first > 1) {
                uint32_t mid = rg.first + (rg.second - rg.first) / 2;
                retry.emplace_back(rg.first, mid);
                retry.emplace_back(mid, rg.second);
                continue;
            }
            // one item alone exceeds the buffer: enlarge it
            dev_free(dbuf[0], s);
            bufcap = cnt;
            SJ_R(dev_alloc(err, dbuf[0], bufcap * 8, s));
            if (sink.cb) {
                pinned_cache().put(stage[0], stage_bytes[0]);
                stage[0] = pinned_cache().get(bufcap * 8, &stage_bytes[0]);
                if (!stage[0]) { cleanup(); return fail(err, SJ_ENOMEM, "pinned host allocation failed"); }
            }
            retry.push_back(rg);
            continue;
        }
        ctx->stats.evaluations += r3[1];
        ctx->stats.rechecks += r3[2];
        ctx->stats.pairs += cnt;
        if (sink.cb) {
            SJ_RC(cudaMemcpyAsync(stage[0], dbuf[0].p, cnt * 8, cudaMemcpyDeviceToHost, s));
            SJ_RC(cudaStreamSynchronize(s));
            if (cnt && sink.cb(static_cast<const uint32_t *>(stage[0]), cnt, sink.user) != 0) sink.stop = true;
        } else {
            sj_result *r = sink.res;
            SJ_R(grow_result(err, r, r->count + cnt));
            SJ_RC(cudaMemcpyAsync(r->pairs + 2 * r->count, dbuf[0].p, cnt * 8, cudaMemcpyDeviceToHost, s));
            SJ_RC(cudaStreamSynchronize(s));
            r->count += cnt;
        }
    }
    cleanup();
#undef SJ_R
#undef SJ_RC
    return SJ_OK;
}

}  // namespace

// Sorts the pairs of a host result ascending by (i << 32) | j on all cores.
void sort_result(sj_result *r) {
    uint64_t *k = reinterpret_cast<uint64_t *>(r->pairs);
    const uint64_t n = r->count;
    // a pair (i, j) read as a little-endian u64 is (j << 32) | i: swap halves
    auto swap_halves = [](uint64_t x) { return (x << 32) | (x >> 32); };
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < (1u << 16)) nt = 1;
    std::vector<std::thread> th;
    std::vector<uint64_t> cut(nt + 1);
    for (unsigned t = 0; t <= nt; ++t) cut[t] = n * t / nt;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (uint64_t i = cut[t]; i < cut[t + 1]; ++i) k[i] = swap_halves(k[i]);
            std::sort(k + cut[t], k + cut[t + 1]);
        });
    for (auto &x : th) x.join();
    for (unsigned w = 1; w < nt; w *= 2) {
        std::vector<std::thread> mt;
        for (unsigned t = 0; t + w < nt; t += 2 * w) {
            uint64_t a = cut[t], m = cut[t + w], e = cut[std::min(nt, t + 2 * w)];
            mt.emplace_back([=]() { std::inplace_merge(k + a, k + m, k + e); });
        }
        for (auto &x : mt) x.join();
    }
    for (uint64_t i = 0; i < n; ++i) k[i] = swap_halves(k[i]);
}

namespace {

sj_status host_join(Error &err, sj_ctx *ctx, Index &ix, HostSink &sink) {
    if (!(ctx->cfg.prec == SJ_PREC_FP32_RECHECK && ix.g.fp32_ok))
        SJ_TRY(ensure_rec64(err, ix, ctx->s_main));
    SJ_TRY(prepare_launch(err, ctx, ix, ctx->s_main));
    SJ_TRY(run_batches(err, ctx, ix, sink));
    record_launch(ctx, ix);
    if (sink.res && ctx->cfg.sorted) sort_result(sink.res);
    return SJ_OK;
}

void reset_stats(sj_ctx *ctx) {
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.frame = -1;
}

}  // namespace
}  // namespace sj

using namespace sj;

extern "C" {

void sj_config_default(sj_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->prec = SJ_PREC_FP32_RECHECK;
    cfg->unicomp = 1;
    cfg->out_cap_bytes = 2ull << 30;
    cfg->min_batches = 3;
    cfg->sorted = 0;
    cfg->autotune = 1;
    cfg->device = 0;
    cfg->lookup = SJ_LOOKUP_AUTO;
    cfg->profile = 0;
    cfg->max_inflight = 64;
    cfg->serve_mem_bytes = 8ull << 30;
    cfg->grab = -1;
    cfg->nbuf = -1;
    cfg->staging = -1;
    cfg->wpb = -1;
    cfg->slots = -1;
    cfg->frame = SJ_FRAME_AUTO;
}

const char *sj_status_str(sj_status st) {
    switch (st) {
        case SJ_OK: return "SJ_OK";
        case SJ_PENDING: return "SJ_PENDING";
        case SJ_EINVAL: return "SJ_EINVAL";
        case SJ_ENOMEM: return "SJ_ENOMEM";
        case SJ_ERANGE: return "SJ_ERANGE";
        case SJ_ECUDA: return "SJ_ECUDA";
        case SJ_ETIMEOUT: return "SJ_ETIMEOUT";
        case SJ_EBUSY: return "SJ_EBUSY";
        case SJ_EOVERFLOW: return "SJ_EOVERFLOW";
        case SJ_ENOTFOUND: return "SJ_ENOTFOUND";
    }
    return "SJ_UNKNOWN";
}

sj_status sj_create(const sj_config *cfg, sj_ctx **out) {
    if (!out) return SJ_EINVAL;
    *out = nullptr;
    sj_config c;
    sj_config_default(&c);
    if (cfg) c = *cfg;
    if (c.prec != SJ_PREC_FP64 && c.prec != SJ_PREC_FP32_RECHECK) return SJ_EINVAL;
    if (c.lookup < SJ_LOOKUP_AUTO || c.lookup > SJ_LOOKUP_COORDS) return SJ_EINVAL;
    if (c.frame < SJ_FRAME_AUTO || c.frame > SJ_FRAME_CELL) return SJ_EINVAL;
    if (c.wait_ms < 0) return SJ_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return SJ_ECUDA;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return SJ_ECUDA;
    sj_ctx *ctx = new sj_ctx();
    ctx->cfg = c;
    ctx->device = c.device;
    ctx->t0 = now_ms();
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->launch = sj::default_launch(ctx);
    Error err;
    // keep freed pool memory cached across calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaStreamCreateWithFlags(&ctx->s_main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
        dev_alloc(err, ctx->misc, kMiscWords * sizeof(unsigned long long), ctx->s_main) != SJ_OK ||
        cudaHostAlloc((void **)&ctx->h_misc, 64 * sizeof(unsigned long long), cudaHostAllocPortable) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_counts, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        sj_destroy(ctx);
        return SJ_ENOMEM;
    }
    cudaStreamSynchronize(ctx->s_main);
    *out = ctx;
    return SJ_OK;
}

void sj_serve_shutdown(sj_ctx *ctx);

void sj_destroy(sj_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    sj_serve_shutdown(ctx);
    if (ctx->s_main) cudaStreamSynchronize(ctx->s_main);
    if (ctx->s_copy) cudaStreamSynchronize(ctx->s_copy);
    dev_free(ctx->misc, ctx->s_main);
    if (ctx->s_main) cudaStreamSynchronize(ctx->s_main);
    if (ctx->h_misc) cudaFreeHost(ctx->h_misc);
    if (ctx->ev_counts) cudaEventDestroy(ctx->ev_counts);
    for (auto &e : ctx->prof) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    if (ctx->s_main) cudaStreamDestroy(ctx->s_main);
    if (ctx->s_copy) cudaStreamDestroy(ctx->s_copy);
    delete ctx;
}

const char *sj_last_error(const sj_ctx *ctx) { return ctx ? ctx->last_err.c_str() : ""; }

sj_status sj_build_index(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                         sj_index **out) {
    if (!ctx || !out) return SJ_EINVAL;
    Scoped sc(ctx);
    *out = nullptr;
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    sj_index *ix = new sj_index();
    ix->device = ctx->device;
    double t0 = now_ms();
    st = build_index(sc.err, pts, n, d, eps, ctx->cfg.lookup, ctx->cfg.frame, ctx->s_main, ix->ix);
    if (st == SJ_OK && ctx->cfg.prec == SJ_PREC_FP64) st = ensure_rec64(sc.err, ix->ix, ctx->s_main);
    if (st == SJ_OK) st = read_counts(sc.err, ix->ix, ctx->s_main);
    if (st != SJ_OK) {
        free_index(ix->ix, ctx->s_main);
        cudaStreamSynchronize(ctx->s_main);
        delete ix;
        return sc.done(st);
    }
    ctx->stats.ms_index = now_ms() - t0;
    ix->ix.owner_stream = nullptr;
    *out = ix;
    return sc.done(SJ_OK);
}

void sj_index_free(sj_index *ix) {
    if (!ix) return;
    cudaSetDevice(ix->device);
    cudaDeviceSynchronize();
    free_index(ix->ix, nullptr);
    cudaDeviceSynchronize();
    delete ix;
}

sj_status sj_index_info(const sj_index *ix, sj_index_desc *out) {
    if (!ix || !out) return SJ_EINVAL;
    std::memset(out, 0, sizeof(*out));
    const Index &x = ix->ix;
    out->n = x.g.n;
    out->d = x.dfull > kMaxDim ? x.dfull : x.g.d;
    out->grid_d = x.g.d;
    for (int j = 0; j < x.g.d; ++j) out->grid_dim[j] = x.dfull > kMaxDim ? x.gdim[j] : j;
    out->dense = x.dense;
    out->eps = x.g.eps;
    out->cell_width = x.g.w;
    out->n_cells = x.n_cells;
    out->grid_cells = x.g.grid_cells;
    for (int j = 0; j < x.g.d; ++j) {
        out->gmin[j] = x.g.gmin[j];
        out->gmax[j] = x.g.gmax[j];
        out->ng[j] = x.g.ng[j];
    }
    out->device_bytes = x.bytes;
    out->fp32 = x.g.fp32_ok;
    out->frame = x.g.frame;
    return SJ_OK;
}

sj_status sj_index_export(const sj_index *ix, uint64_t *B, uint32_t *G, uint32_t *A, uint32_t *M) {
    if (!ix) return SJ_EINVAL;
    const Index &x = ix->ix;
    cudaSetDevice(ix->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (B && !x.B.p) return SJ_ERANGE;   // cells ordered by coordinate tuple: no linear ids
    if (e == cudaSuccess && B) e = cudaMemcpy(B, x.B.p, x.n_cells * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && G) e = cudaMemcpy(G, x.G.p, (x.n_cells + 1) * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && A) e = cudaMemcpy(A, x.A.p, x.g.n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && M)
        e = cudaMemcpy(M, x.M.p, (size_t)x.g.d * x.mwords * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SJ_OK : SJ_ECUDA;
}

static sj_status device_join_on(sj_ctx *ctx, Error &err, Index &ix, uint32_t *d_pairs,
                                uint64_t cap, uint64_t *count, cudaStream_t s, int count_only,
                                uint32_t item_begin = 0, uint32_t item_end = 0xffffffffu) {
    if (!(ctx->cfg.prec == SJ_PREC_FP32_RECHECK && ix.g.fp32_ok)) SJ_TRY(ensure_rec64(err, ix, s));
    SJ_TRY(prepare_launch(err, ctx, ix, s));
    unsigned long long r[3];
    SJ_TRY(join_once(err, ctx, ix, item_begin, item_end, 1, reinterpret_cast<uint2 *>(d_pairs), cap,
                     count_only, s, r));
    *count = r[0];
    record_launch(ctx, ix);
    ctx->stats.pairs = r[0];
    ctx->stats.evaluations = r[1];
    ctx->stats.rechecks = r[2];
    ctx->stats.batches = 1;
    if (!count_only && r[0] > cap)
        return fail(err, SJ_EOVERFLOW, "output buffer too small for the pair count");
    return SJ_OK;
}

sj_status sj_selfjoin_device(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                             uint32_t *d_pairs, uint64_t cap_pairs, uint64_t *count, void *stream) {
    if (!ctx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if (!d_pairs && cap_pairs) return sc.done(fail(sc.err, SJ_EINVAL, "d_pairs is NULL"));
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double t0 = now_ms();
    const BuildOpts bo = call_build_opts(ctx);
    Index ix;
    st = build_index(sc.err, pts, n, d, eps, ctx->cfg.lookup, ctx->cfg.frame, s, ix, nullptr, &bo);
    double t1 = now_ms();
    if (st == SJ_OK) st = device_join_on(ctx, sc.err, ix, d_pairs, cap_pairs, count, s, 0);
    free_index(ix, s);
    ctx->stats.ms_index = t1 - t0;
    ctx->stats.ms_join = now_ms() - t1;
    ctx->stats.ms_total = now_ms() - t0;
    return sc.done(st);
}

sj_status sj_selfjoin_shard_device(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                                   int rank, int world, uint32_t *d_pairs, uint64_t cap_pairs,
                                   uint64_t *count, void *stream) {
    if (!ctx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if (world < 1 || rank < 0 || rank >= world)
        return sc.done(fail(sc.err, SJ_EINVAL, "rank must be in [0, world)"));
    if (!d_pairs && cap_pairs) return sc.done(fail(sc.err, SJ_EINVAL, "d_pairs is NULL"));
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double t0 = now_ms();
    const BuildOpts bo = call_build_opts(ctx);
    Index ix;
    st = build_index(sc.err, pts, n, d, eps, ctx->cfg.lookup, ctx->cfg.frame, s, ix, nullptr, &bo);
    double t1 = now_ms();
    uint32_t lo = 0, hi = 0;
    if (st == SJ_OK) st = shard_items(sc.err, ix, ctx->cfg.unicomp != 0, rank, world, s, &lo, &hi);
    if (st == SJ_OK) st = device_join_on(ctx, sc.err, ix, d_pairs, cap_pairs, count, s, 0, lo, hi);
    free_index(ix, s);
    ctx->stats.ms_index = t1 - t0;
    ctx->stats.ms_join = now_ms() - t1;
    ctx->stats.ms_total = now_ms() - t0;
    return sc.done(st);
}

sj_status sj_join2_device(sj_ctx *ctx, const double *R, uint64_t nR, const double *S, uint64_t nS,
                          int d, double eps, uint32_t *d_pairs, uint64_t cap_pairs, uint64_t *count,
                          void *stream) {
    if (!ctx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, R, nR, d, eps);
    if (st == SJ_OK) st = check_args(sc.err, S, nS, d, eps);
    if (st == SJ_OK && d > kMaxDim) st = fail(sc.err, SJ_EINVAL, "two-set joins take at most 8 dimensions");
    if (st != SJ_OK) return sc.done(st);
    if (!d_pairs && cap_pairs) return sc.done(fail(sc.err, SJ_EINVAL, "d_pairs is NULL"));
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Error &err = sc.err;
    const double t0 = now_ms();
    DevBuf dR, dS;
    Index ixR, ixS;
    auto run = [&]() -> sj_status {
        // one grid over both sets (Section IV-B on the union bounding box)
        SJ_TRY(dev_alloc(err, dR, nR * d * sizeof(double), s));
        SJ_TRY(dev_alloc(err, dS, nS * d * sizeof(double), s));
        SJ_CUDA_TRY(cudaMemcpyAsync(dR.p, R, nR * d * sizeof(double), cudaMemcpyDefault, s));
        SJ_CUDA_TRY(cudaMemcpyAsync(dS.p, S, nS * d * sizeof(double), cudaMemcpyDefault, s));
        unsigned long long mR[2 * kMaxDim], mS[2 * kMaxDim], mm[2 * kMaxDim] = {0};
        bool badR = false, badS = false;
        SJ_TRY(bounds_of(err, static_cast<const double *>(dR.p), nR, d, s, mR, &badR));
        SJ_TRY(bounds_of(err, static_cast<const double *>(dS.p), nS, d, s, mS, &badS));
        if (badR || badS) return fail(err, SJ_EINVAL, "non-finite coordinate");
        for (int j = 0; j < d; ++j) {
            mm[2 * j] = std::min(mR[2 * j], mS[2 * j]);
            mm[2 * j + 1] = std::max(mR[2 * j + 1], mS[2 * j + 1]);
        }
        BuildOpts bo_in;
        bo_in.borrow_pts = true;
        SJ_TRY(build_index(err, static_cast<const double *>(dS.p), nS, d, eps, ctx->cfg.lookup, ctx->cfg.frame, s, ixS, mm, &bo_in));
        SJ_TRY(build_index(err, static_cast<const double *>(dR.p), nR, d, eps, ctx->cfg.lookup, ctx->cfg.frame, s, ixR, mm, &bo_in));
        const double t1 = now_ms();
        ctx->stats.ms_index = t1 - t0;
        JoinLaunch l = default_launch(ctx);
        l.unicomp = 0;   // R and S differ: every query searches all adjacent cells
        ctx->stats.frame = (l.prec_fp32 && ixS.g.fp32_ok) ? ixS.g.frame : -1;
        if (!(l.prec_fp32 && ixS.g.fp32_ok)) {
            SJ_TRY(ensure_rec64(err, ixS, s));
            SJ_TRY(ensure_rec64(err, ixR, s));
        }
        unsigned long long *m = misc_dev(ctx);
        SJ_CUDA_TRY(cudaMemsetAsync(m, 0, kMiscWords * sizeof(unsigned long long), s));
        cudaEvent_t e0, e1;
        SJ_TRY(profile_events(err, ctx, &e0, &e1));
        SJ_TRY(launch_join(err, ixS, l, 0, 0xffffffffu, reinterpret_cast<uint2 *>(d_pairs), cap_pairs,
                           m + kMiscCounter, reinterpret_cast<uint32_t *>(m + kMiscWork),
                           reinterpret_cast<uint32_t *>(m + kMiscError), 0, s, e0, e1, &ixR));
        SJ_CUDA_TRY(cudaMemcpyAsync(ctx->h_misc, m, kMiscWords * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        if ((uint32_t)ctx->h_misc[kMiscError] & kErrTimeout)
            return fail(err, SJ_ETIMEOUT, "a bounded device wait expired in the join kernel");
        *count = ctx->h_misc[0];
        ctx->stats.pairs = ctx->h_misc[0];
        ctx->stats.evaluations = ctx->h_misc[1];
        ctx->stats.rechecks = ctx->h_misc[2];
        ctx->stats.batches = 1;
        ctx->stats.ms_join = now_ms() - t1;
        return SJ_OK;
    };
    st = run();
    free_index(ixR, s);
    free_index(ixS, s);
    dev_free(dR, s);
    dev_free(dS, s);
    ctx->stats.ms_total = now_ms() - t0;
    if (st == SJ_OK && *count > cap_pairs)
        st = fail(err, SJ_EOVERFLOW, "output buffer too small for the pair count");
    return sc.done(st);
}

sj_status sj_selfjoin_bruteforce_device(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                                        uint32_t *d_pairs, uint64_t cap_pairs, uint64_t *count,
                                        void *stream) {
    if (!ctx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if (!d_pairs && cap_pairs) return sc.done(fail(sc.err, SJ_EINVAL, "d_pairs is NULL"));
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double t0 = now_ms();
    Error &err = sc.err;
    DevBuf dp;
    auto run = [&]() -> sj_status {
        SJ_TRY(dev_alloc(err, dp, n * d * sizeof(double), s));
        SJ_CUDA_TRY(cudaMemcpyAsync(dp.p, pts, n * d * sizeof(double), cudaMemcpyDefault, s));
        unsigned long long *m = misc_dev(ctx);
        SJ_CUDA_TRY(cudaMemsetAsync(m, 0, kMiscWords * sizeof(unsigned long long), s));
        SJ_TRY(brute_join(err, static_cast<const double *>(dp.p), n, d, eps,
                          reinterpret_cast<uint2 *>(d_pairs), cap_pairs, m + kMiscCounter, s));
        SJ_CUDA_TRY(cudaMemcpyAsync(ctx->h_misc, m, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        SJ_CUDA_TRY(cudaStreamSynchronize(s));
        return SJ_OK;
    };
    st = run();
    dev_free(dp, s);
    if (st == SJ_OK) {
        *count = ctx->h_misc[0];
        ctx->stats.pairs = *count;
        ctx->stats.evaluations = n * n;
        ctx->stats.batches = 1;
        ctx->stats.ms_total = now_ms() - t0;
        if (*count > cap_pairs) st = fail(err, SJ_EOVERFLOW, "output buffer too small for the pair count");
    }
    return sc.done(st);
}

sj_status sj_selfjoin_index_device(sj_ctx *ctx, const sj_index *idx, uint32_t *d_pairs,
                                   uint64_t cap_pairs, uint64_t *count, void *stream) {
    if (!ctx || !idx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    if (!d_pairs && cap_pairs) return sc.done(fail(sc.err, SJ_EINVAL, "d_pairs is NULL"));
    sj_status st = set_device(sc.err, ctx->device);
    if (st != SJ_OK) return sc.done(st);
    double t0 = now_ms();
    st = device_join_on(ctx, sc.err, const_cast<sj_index *>(idx)->ix, d_pairs, cap_pairs, count,
                        static_cast<cudaStream_t>(stream), 0);
    ctx->stats.ms_join = ctx->stats.ms_total = now_ms() - t0;
    return sc.done(st);
}

sj_status sj_selfjoin_count(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                            uint64_t *count) {
    if (!ctx || !count) return SJ_EINVAL;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    double t0 = now_ms();
    const BuildOpts bo = call_build_opts(ctx);
    Index ix;
    st = build_index(sc.err, pts, n, d, eps, ctx->cfg.lookup, ctx->cfg.frame, ctx->s_main, ix, nullptr, &bo);
    if (st == SJ_OK) st = device_join_on(ctx, sc.err, ix, nullptr, 0, count, ctx->s_main, 1);
    free_index(ix, ctx->s_main);
    cudaStreamSynchronize(ctx->s_main);
    ctx->stats.ms_total = now_ms() - t0;
    return sc.done(st);
}

static sj_status host_join_from_pts(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                                    HostSink &sink) {
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = check_args(sc.err, pts, n, d, eps);
    if (st != SJ_OK) return sc.done(st);
    if ((st = set_device(sc.err, ctx->device)) != SJ_OK) return sc.done(st);
    double t0 = now_ms();
    const BuildOpts bo = call_build_opts(ctx);
    Index ix;
    st = build_index(sc.err, pts, n, d, eps, ctx->cfg.lookup, ctx->cfg.frame, ctx->s_main, ix, nullptr, &bo);
    double t1 = now_ms();
    if (st == SJ_OK) st = host_join(sc.err, ctx, ix, sink);
    free_index(ix, ctx->s_main);
    cudaStreamSynchronize(ctx->s_main);
    ctx->stats.ms_index = t1 - t0;
    ctx->stats.ms_join = now_ms() - t1;
    ctx->stats.ms_total = now_ms() - t0;
    if (sink.res) ctx->stats.pairs = sink.res->count;
    ctx->stats.n_cells = ix.n_cells;
    return sc.done(st);
}

sj_status sj_selfjoin(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                      sj_result **out) {
    if (!ctx || !out) return SJ_EINVAL;
    *out = nullptr;
    sj_result *r = new sj_result();
    HostSink sink;
    sink.res = r;
    sj_status st = host_join_from_pts(ctx, pts, n, d, eps, sink);
    if (st != SJ_OK) { sj_result_free(r); return st; }
    *out = r;
    return SJ_OK;
}

sj_status sj_selfjoin_index(sj_ctx *ctx, const sj_index *idx, sj_result **out) {
    if (!ctx || !idx || !out) return SJ_EINVAL;
    *out = nullptr;
    Scoped sc(ctx);
    reset_stats(ctx);
    sj_status st = set_device(sc.err, ctx->device);
    if (st != SJ_OK) return sc.done(st);
    sj_result *r = new sj_result();
    HostSink sink;
    sink.res = r;
    double t0 = now_ms();
    st = host_join(sc.err, ctx, const_cast<sj_index *>(idx)->ix, sink);
    ctx->stats.ms_join = ctx->stats.ms_total = now_ms() - t0;
    ctx->stats.pairs = r->count;
    if (st != SJ_OK) { sj_result_free(r); return sc.done(st); }
    *out = r;
    return sc.done(SJ_OK);
}

sj_status sj_selfjoin_stream(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps,
                             sj_chunk_cb cb, void *user) {
    if (!ctx || !cb) return SJ_EINVAL;
    HostSink sink;
    sink.cb = cb;
    sink.user = user;
    return host_join_from_pts(ctx, pts, n, d, eps, sink);
}

uint64_t sj_result_count(const sj_result *r) { return r ? r->count : 0; }
const uint32_t *sj_result_pairs(const sj_result *r) { return r ? r->pairs : nullptr; }

void sj_result_free(sj_result *r) {
    if (!r) return;
    if (r->pairs) pinned_cache().put(r->pairs, r->bytes);
    delete r;
}

sj_status sj_result_times(const sj_result *r, double *t_submit, double *t_admit, double *t_done) {
    if (!r) return SJ_EINVAL;
    if (t_submit) *t_submit = r->t_submit;
    if (t_admit) *t_admit = r->t_admit;
    if (t_done) *t_done = r->t_done;
    return SJ_OK;
}

void sj_tune_reset(void) {
    tune_clear();
    engine_tune_reset();
}

sj_status sj_last_stats(const sj_ctx *ctx, sj_stats *out) {
    if (!ctx || !out) return SJ_EINVAL;
    *out = ctx->stats;
    return SJ_OK;
}

sj_status sj_profile_read(sj_ctx *ctx, double *kernel_ms, uint64_t *launches) {
    if (!ctx) return SJ_EINVAL;
    cudaSetDevice(ctx->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return SJ_ECUDA;
    double ms = 0;
    for (size_t i = 0; i < ctx->prof_used; ++i) {
        float f = 0;
        if (cudaEventElapsedTime(&f, ctx->prof[i].first, ctx->prof[i].second) == cudaSuccess) ms += f;
        else cudaGetLastError();
    }
    if (kernel_ms) *kernel_ms = ms;
    if (launches) *launches = ctx->prof_used;
    ctx->prof_used = 0;
    return SJ_OK;
}

}  // extern "C"
