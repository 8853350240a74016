// tune.cu -- launch tuner of the search-and-refine kernel.
//
// Five launch parameters change the speed of the join but never its
// result: grab (the work items a warp takes from the cursor at a time: how
// many (cell, query block) items it owns before it returns for more), the
// depth of the per-warp ring of staged candidate chunks, the item slots per
// warp (preparing the next item ahead against shared memory), the size of
// the per-warp pair staging area (few large flushes when hits are dense, as
// in clustered data, against more resident warps), and the warps per block
// (which trades shared memory per block against blocks per SM).  Their
// best values depend on the dimension, the precision and how many points a
// non-empty cell holds (few per cell: short candidate lists, latency-bound
// copies; many per cell, as in clustered data: long lists, skew between
// items).  The tuner keys its choices on (d, precision, UNICOMP, bucket)
// with bucket = round(log2(mean points per non-empty cell)), and on a miss
// times launches of the join at hand over a fixed systematic sample of its
// work items (the same items for every candidate; the sample's pairs are
// written to a scratch buffer when it fits in 512 MB, else counted only),
// one parameter after the other, keeping a change only when it is at least
// 3% faster.  Choices are kept for the life of the process.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "sj_internal.cuh"

namespace sj {

namespace {

struct TuneVal {
    int grab = 1, nbuf = 0, wpb = 0, eb = 0, slots = 0;
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TuneVal> g_tune;

constexpr uint32_t kTuneSampleItems = 24576;  // items per timed launch
constexpr uint64_t kTuneMaxOutBytes = 512ull << 20;  // above: time count-only launches

}  // namespace

bool launch_forced(const sj_config &c) {
    return c.grab > 0 || c.nbuf > 0 || c.staging > 0 || c.wpb > 0 || c.slots > 0;
}

int tune_bucket_ppc(double points_per_cell) {
    return (int)std::lround(std::log2(std::max(1.0, points_per_cell)));
}

int tune_bucket(const Index &ix) {
    return tune_bucket_ppc(ix.n_cells ? (double)ix.g.n / (double)ix.n_cells : 1.0);
}

sj_status tune_launch(Error &err, Index &ix, JoinLaunch &l, cudaStream_t s, int *tuned) {
    *tuned = 0;
    const bool f32 = l.prec_fp32 && ix.g.fp32_ok;
    const auto key = std::make_tuple(ix.g.d, f32 ? 1 : 0, l.unicomp ? 1 : 0, tune_bucket(ix));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            l.grab = it->second.grab;
            l.nbuf = it->second.nbuf;
            l.wpb = it->second.wpb;
            l.eb = it->second.eb;
            l.slots = it->second.slots;
            *tuned = 1;
            return SJ_OK;
        }
    }
    SJ_TRY(read_counts(err, ix, s));   // a miss needs the work-item count
    if (ix.n_items < kTuneMinItems) return SJ_OK;
    DevBuf misc;
    SJ_TRY(dev_alloc(err, misc, 64, s));
    unsigned long long *m = static_cast<unsigned long long *>(misc.p);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sj_status st = SJ_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = fail(err, SJ_ECUDA, "cudaEventCreate failed");
    }
    uint32_t stride = std::max<uint32_t>(1, ix.n_items / kTuneSampleItems);
    // the sample's pair count, so that the timed launches can write their
    // pairs (the staging size only matters with the stores); a sample whose
    // pairs exceed kTuneMaxOutBytes is thinned until they fit
    DevBuf outb;
    uint64_t sample_pairs = 0;
    auto count_sample = [&](uint32_t str, uint64_t *pairs) -> sj_status {
        JoinLaunch x = l;
        x.item_stride = str;
        unsigned long long h[8] = {0};
        if (cudaMemsetAsync(m, 0, 64, s) != cudaSuccess ||
            launch_join(err, ix, x, 0, ix.n_items, nullptr, 0, m, reinterpret_cast<uint32_t *>(m + 4),
                        reinterpret_cast<uint32_t *>(m + 5), 1, s, nullptr, nullptr) != SJ_OK ||
            cudaMemcpyAsync(h, m, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return err.st != SJ_OK ? err.st : fail(err, SJ_ECUDA, "tuner sample count failed");
        }
        *pairs = h[0];
        return SJ_OK;
    };
    if (st == SJ_OK) st = count_sample(stride, &sample_pairs);
    for (int tries = 0; st == SJ_OK && sample_pairs * 8 > kTuneMaxOutBytes && tries < 4; ++tries) {
        const uint64_t f = (sample_pairs * 8 + kTuneMaxOutBytes - 1) / kTuneMaxOutBytes;
        if ((uint64_t)stride * f * 64 > ix.n_items) break;   // keep at least 64 items
        stride = (uint32_t)(stride * f);
        st = count_sample(stride, &sample_pairs);
    }
    if (st == SJ_OK && sample_pairs * 8 <= kTuneMaxOutBytes) {
        Error e2;
        if (dev_alloc(e2, outb, std::max<uint64_t>(sample_pairs, 1) * 8, s) != SJ_OK) outb = DevBuf();
    }
    const int count_only = outb.p ? 0 : 1;
    auto time_it = [&](const JoinLaunch &c, double *ms) -> sj_status {
        JoinLaunch x = c;
        x.item_stride = stride;
        double best = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            SJ_CUDA_TRY(cudaMemsetAsync(m, 0, 64, s));
            SJ_TRY(launch_join(err, ix, x, 0, ix.n_items, static_cast<uint2 *>(outb.p),
                               outb.p ? sample_pairs : 0, m, reinterpret_cast<uint32_t *>(m + 4),
                               reinterpret_cast<uint32_t *>(m + 5), count_only, s, e0, e1));
            SJ_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0;
            SJ_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, (double)t);
        }
        unsigned long long h[8];
        SJ_CUDA_TRY(cudaMemcpy(h, m, sizeof(h), cudaMemcpyDeviceToHost));
        if ((uint32_t)h[5] & kErrTimeout) return fail(err, SJ_ETIMEOUT, "a bounded device wait expired while tuning");
        *ms = best;
        return SJ_OK;
    };
    JoinLaunch cur = l;
    if (cur.grab <= 0) cur.grab = 1;
    double t_cur = 0;
    if (st == SJ_OK) st = time_it(cur, &t_cur);
    const int grabs[] = {2, 4, 8, 16};
    const int nbufs[] = {2, 3, 4, 6};
    const int wpbs[] = {8, 4, 2};
    for (int g : grabs) {
        if (st != SJ_OK) break;
        JoinLaunch c = cur;
        c.grab = g;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) { cur = c; t_cur = t; }
    }
    for (int nb : nbufs) {
        if (st != SJ_OK) break;
        JoinLaunch c = cur;
        c.nbuf = nb;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) { cur = c; t_cur = t; }
    }
    const int slotss[] = {1, 2};
    for (int sl : slotss) {
        if (st != SJ_OK) break;
        JoinLaunch c = cur;
        c.slots = sl;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) { cur = c; t_cur = t; }
    }
    const int ebs[] = {256, 512, 1024};
    for (int eb : ebs) {
        if (st != SJ_OK) break;
        JoinLaunch c = cur;
        c.eb = eb;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) { cur = c; t_cur = t; }
    }
    for (int w : wpbs) {
        if (st != SJ_OK) break;
        JoinLaunch c = cur;
        c.wpb = w;
        double t = 0;
        st = time_it(c, &t);
        if (st == SJ_OK && t < 0.97 * t_cur) { cur = c; t_cur = t; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(outb, s);
    dev_free(misc, s);
    if (st != SJ_OK) return st;
    TuneVal v;
    v.grab = cur.grab;
    v.nbuf = cur.nbuf;
    v.wpb = cur.wpb;
    v.eb = cur.eb;
    v.slots = cur.slots;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = v;
    }
    l.grab = v.grab;
    l.nbuf = v.nbuf;
    l.wpb = v.wpb;
    l.eb = v.eb;
    l.slots = v.slots;
    *tuned = 2;
    return SJ_OK;
}

void tune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // namespace sj
