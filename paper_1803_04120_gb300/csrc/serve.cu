// serve.cu -- the request interface of include/sj.h: continuous batching of
// join requests (sj_submit / sj_poll) and the multi-join call
// sj_selfjoin_multi.
//
// Scheduler.  sj_submit copies the request's points into pinned host memory,
// estimates the device bytes the request will hold (points, index, result
// buffer; engine.cu) and queues it.  Each of kLanes lane threads owns a
// multi-join engine (its own stream, job tables and CUDA graph).  An idle
// lane admits queued requests in arrival order and runs them as one wave,
// while all of these hold:
//   - fewer than max_inflight requests are admitted over all lanes;
//   - the admitted estimated bytes fit in serve_mem_bytes;
//   - the wave has at most kMultiJobs requests, and no more estimated
//     pairs than kWavePairs beyond its first request.
// Each request is handed out as soon as its own pairs are on the host,
// smaller results first; its memory estimate and slot are returned then.
// So requests that arrive while a wave runs are admitted by another lane
// as soon as slots and memory allow, and the waves overlap on the device.  A request's result does not depend on the wave it ran in: every
// job has its own index, cursor, counters and output.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "engine.cuh"

namespace {

using namespace sj;

// Lanes: a lane alternates host work (points in, bounds read-back), the
// graph and the copy-out of its wave, so with two lanes the device-to-host
// link (the serving bound) idles whenever neither is copying.  Measured on
// the 10,000-request stream: 10.7, 11.6 and 12.1 G pairs/s saturated with
// 2, 3 and 4 lanes.
constexpr int kLanes = 4;

struct Request {
    uint64_t ticket = 0;
    double *pts = nullptr;      // pinned copy of the points
    size_t pts_bytes = 0;
    uint64_t n = 0;
    int d = 0;
    double eps = 0;
    uint64_t est_bytes = 0;
    uint64_t est_pairs = 0;
    double t_submit = 0, t_admit = 0;
};

// Estimated pairs one wave may hold beyond its first request: a very large
// request then runs in a wave of its own while the other lane keeps
// serving the small ones.
constexpr uint64_t kWavePairs = 250000000ull;

struct Finished {
    sj_status st = SJ_OK;
    sj_result *r = nullptr;
};

struct Server {
    sj_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Finished> done;
    std::unordered_set<uint64_t> pending;    // queued or running
    uint64_t next_ticket = 1;
    uint64_t mem_in_use = 0;
    int inflight = 0;
    int running_waves = 0;
    bool stop = false;
    std::vector<std::thread> lanes;
    std::vector<Engine *> engines;
    sj_serve_info info;
};

std::mutex g_serve_mu;   // creation and shutdown of servers

double secs(const sj_ctx *ctx) { return (now_ms() - ctx->t0) / 1000.0; }

int max_inflight(const sj_ctx *ctx) { return ctx->cfg.max_inflight > 0 ? ctx->cfg.max_inflight : 64; }

uint64_t mem_budget(const sj_ctx *ctx) {
    return ctx->cfg.serve_mem_bytes > 0 ? ctx->cfg.serve_mem_bytes : (8ull << 30);
}

bool admissible(const Server *S) {
    if (S->queue.empty() || S->inflight >= max_inflight(S->ctx)) return false;
    return S->inflight == 0 || S->mem_in_use + S->queue.front().est_bytes <= mem_budget(S->ctx);
}

// Hands out a finished request: its result (or error) becomes visible to
// sj_poll and its memory estimate and slot are returned.
void finish(Server *S, Request &r, EngJob &J, sj_status st, double t_done) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        Finished f;
        f.st = st;
        f.r = st == SJ_OK ? J.res : nullptr;
        if (st != SJ_OK && J.res) sj_result_free(J.res);
        J.res = nullptr;
        if (f.r) {
            f.r->t_submit = r.t_submit;
            f.r->t_admit = r.t_admit;
            f.r->t_done = t_done;
        }
        S->done[r.ticket] = f;
        S->pending.erase(r.ticket);
        S->mem_in_use -= r.est_bytes;
        S->inflight--;
        S->info.completed++;
        if (J.path == 2) S->info.overflow_reruns++;
        if (J.path == 1) S->info.standalone++;
        pinned_put(r.pts, r.pts_bytes);
        r.pts = nullptr;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

struct WaveState {
    Server *S;
    std::vector<Request> *wave;
    std::vector<EngJob> *jobs;
    std::vector<char> done;
};

void on_job_done(void *user, int q) {
    WaveState *w = static_cast<WaveState *>(user);
    if (w->done[q]) return;
    w->done[q] = 1;
    finish(w->S, (*w->wave)[q], (*w->jobs)[q], (*w->jobs)[q].st, secs(w->S->ctx));
}

void lane_main(Server *S, int lane) {
    cudaSetDevice(S->ctx->device);
    Engine *E = S->engines[lane];
    for (;;) {
        std::vector<Request> wave;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || admissible(S); });
            if (S->stop) break;
            const double t = secs(S->ctx);
            uint64_t pairs = 0;
            while (admissible(S) && (int)wave.size() < kMultiJobs &&
                   (wave.empty() || pairs + S->queue.front().est_pairs <= kWavePairs)) {
                Request r = std::move(S->queue.front());
                S->queue.pop_front();
                r.t_admit = t;
                pairs += r.est_pairs;
                S->mem_in_use += r.est_bytes;
                S->inflight++;
                wave.push_back(std::move(r));
            }
            S->running_waves++;
            S->info.max_concurrent_waves = std::max<int32_t>(S->info.max_concurrent_waves, S->running_waves);
            S->info.waves++;
            S->info.max_wave = std::max<uint64_t>(S->info.max_wave, wave.size());
        }
        // a lane that admitted a wave may leave work for the other lane
        S->cv_work.notify_all();
        std::vector<EngJob> jobs(wave.size());
        std::vector<EngJob *> ptrs;
        for (size_t q = 0; q < wave.size(); ++q) {
            jobs[q].pts = wave[q].pts;
            jobs[q].n = wave[q].n;
            jobs[q].d = wave[q].d;
            jobs[q].eps = wave[q].eps;
            ptrs.push_back(&jobs[q]);
        }
        WaveState ws{S, &wave, &jobs, std::vector<char>(wave.size(), 0)};
        Error err;
        const sj_status st = engine_run(err, E, ptrs.data(), (int)ptrs.size(), on_job_done, &ws);
        // requests the engine did not hand out (it stopped on an error)
        for (size_t q = 0; q < wave.size(); ++q)
            if (!ws.done[q]) {
                ws.done[q] = 1;
                finish(S, wave[q], jobs[q], st != SJ_OK ? st : jobs[q].st, secs(S->ctx));
            }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->running_waves--;
        }
        S->cv_work.notify_all();
    }
}

Server *get_server(sj_ctx *ctx, sj_status *st) {
    std::lock_guard<std::mutex> lk(g_serve_mu);
    *st = SJ_OK;
    if (ctx->serve) return static_cast<Server *>(ctx->serve);
    Server *S = new Server();
    S->ctx = ctx;
    std::memset(&S->info, 0, sizeof(S->info));
    S->info.lanes = kLanes;
    for (int l = 0; l < kLanes; ++l) {
        Error err;
        Engine *E = nullptr;
        const sj_status es = engine_create(err, ctx->device, ctx->cfg, &E);
        if (es != SJ_OK) {
            for (Engine *x : S->engines) engine_destroy(x);
            delete S;
            *st = es;
            return nullptr;
        }
        S->engines.push_back(E);
    }
    for (int l = 0; l < kLanes; ++l) S->lanes.emplace_back(lane_main, S, l);
    ctx->serve = S;
    return S;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sj_status check_job(const double *pts, uint64_t n, int d, double eps) {
    if (!pts || n == 0 || d < 1 || d > kMaxDim || !(eps > 0.0) || !std::isfinite(eps)) return SJ_EINVAL;
    if (n >= (1ull << 32)) return SJ_ERANGE;
    return SJ_OK;
}

}  // namespace

extern "C" {

void sj_serve_shutdown(sj_ctx *ctx) {
    if (!ctx) return;
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_serve_mu);
        S = static_cast<Server *>(ctx->serve);
        ctx->serve = nullptr;
    }
    if (S) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        for (std::thread &t : S->lanes) t.join();
        for (Request &r : S->queue) pinned_put(r.pts, r.pts_bytes);
        for (auto &kv : S->done)
            if (kv.second.r) sj_result_free(kv.second.r);
        for (Engine *E : S->engines) engine_destroy(E);
        delete S;
    }
    if (ctx->engine) {
        engine_destroy(static_cast<Engine *>(ctx->engine));
        ctx->engine = nullptr;
    }
}

sj_status sj_submit(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps, uint64_t *ticket) {
    if (!ctx || !ticket) return SJ_EINVAL;
    *ticket = 0;
    sj_status st = check_job(pts, n, d, eps);
    if (st != SJ_OK) return st;
    const double t_submit = secs(ctx);
    cudaSetDevice(ctx->device);
    Request r;
    r.n = n;
    r.d = d;
    r.eps = eps;
    r.t_submit = t_submit;
    const size_t bytes = (size_t)n * d * sizeof(double);
    r.pts = static_cast<double *>(pinned_get(bytes, &r.pts_bytes));
    if (!r.pts) return SJ_ENOMEM;
    if (is_device_ptr(pts)) {
        if (cudaMemcpy(r.pts, pts, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            pinned_put(r.pts, r.pts_bytes);
            return SJ_ECUDA;
        }
    } else {
        std::memcpy(r.pts, pts, bytes);
    }
    // non-finite coordinates are found by the device bounds pass; the
    // request then finishes with SJ_EINVAL
    r.est_bytes = engine_estimate(r.pts, n, d, eps, &r.est_pairs);
    if (r.est_bytes > mem_budget(ctx)) {
        pinned_put(r.pts, r.pts_bytes);
        return SJ_ENOMEM;
    }
    Server *S = get_server(ctx, &st);
    if (!S) {
        pinned_put(r.pts, r.pts_bytes);
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        S->pending.insert(r.ticket);
        S->queue.push_back(std::move(r));
        S->info.submitted++;
    }
    S->cv_work.notify_one();
    return SJ_OK;
}

sj_status sj_poll(sj_ctx *ctx, uint64_t ticket, int wait_ms, sj_result **out) {
    if (!ctx || !out) return SJ_EINVAL;
    *out = nullptr;
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_serve_mu);
        S = static_cast<Server *>(ctx->serve);
    }
    if (!S) return SJ_ENOTFOUND;
    std::unique_lock<std::mutex> lk(S->mu);
    auto take = [&](sj_status *st) {
        auto it = S->done.find(ticket);
        if (it == S->done.end()) return false;
        *st = it->second.st;
        *out = it->second.r;
        S->done.erase(it);
        return true;
    };
    sj_status st;
    if (take(&st)) return st;
    if (!S->pending.count(ticket)) return SJ_ENOTFOUND;
    if (wait_ms > 0) {
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                            [&] { return S->done.count(ticket) != 0; });
        if (take(&st)) return st;
    }
    return SJ_PENDING;
}

sj_status sj_serve_stats(sj_ctx *ctx, sj_serve_info *out) {
    if (!ctx || !out) return SJ_EINVAL;
    std::memset(out, 0, sizeof(*out));
    Server *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_serve_mu);
        S = static_cast<Server *>(ctx->serve);
    }
    if (!S) return SJ_OK;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->info;
    out->queued = S->queue.size();
    out->inflight = S->inflight;
    out->mem_in_use = S->mem_in_use;
    uint64_t g = 0;
    for (Engine *E : S->engines) {
        const EngStats es = engine_stats(E);
        g += es.graph_launches;
        out->tuned_waves += es.tuned_waves;
        out->ms_tune += es.ms_tune;
        out->ms_bounds += es.ms_bounds;
        out->ms_graph += es.ms_graph;
        out->ms_output += es.ms_output;
    }
    out->graph_launches = g;
    return SJ_OK;
}

sj_status sj_selfjoin_multi(sj_ctx *ctx, const sj_job *jobs, uint64_t n_jobs, sj_result **out,
                            sj_status *status) {
    if (!ctx) return SJ_EINVAL;
    if (n_jobs == 0) return SJ_OK;
    if (!jobs || !out) {
        ctx->last_err = "jobs and out must not be NULL";
        return SJ_EINVAL;
    }
    for (uint64_t i = 0; i < n_jobs; ++i) {
        out[i] = nullptr;
        if (status) status[i] = SJ_PENDING;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return SJ_ECUDA;
    }
    const uint64_t l0 = launches_so_far();
    Error err;
    if (!ctx->engine) {
        Engine *E = nullptr;
        const sj_status es = engine_create(err, ctx->device, ctx->cfg, &E);
        if (es != SJ_OK) {
            ctx->last_err = err.msg;
            return es;
        }
        ctx->engine = E;
    }
    Engine *E = static_cast<Engine *>(ctx->engine);
    const uint64_t budget = mem_budget(ctx);
    sj_status first = SJ_OK;
    std::string first_msg;
    uint64_t pairs = 0, evals = 0, rechecks = 0, waves = 0, reruns = 0;
    int tuned = 0;
    EngStats last;
    const double t0 = now_ms();
    for (uint64_t b = 0; b < n_jobs;) {
        std::vector<EngJob> wave;
        uint64_t bytes = 0;
        while (b < n_jobs && wave.size() < (size_t)kMultiJobs) {
            const sj_job &J = jobs[b];
            uint64_t est = 0;
            if (check_job(J.pts, J.n, J.d, J.eps) == SJ_OK) {
                est = is_device_ptr(J.pts)
                          ? (uint64_t)J.n * (8ull * J.d + 120) + (256ull << 20)
                          : engine_estimate(J.pts, J.n, J.d, J.eps, nullptr);
            }
            if (!wave.empty() && bytes + est > budget) break;
            EngJob e;
            e.pts = J.pts;
            e.n = J.n;
            e.d = J.d;
            e.eps = J.eps;
            wave.push_back(e);
            bytes += est;
            ++b;
        }
        std::vector<EngJob *> ptrs;
        for (EngJob &e : wave) ptrs.push_back(&e);
        const sj_status st = engine_run(err, E, ptrs.data(), (int)ptrs.size());
        ++waves;
        last = engine_stats(E);
        tuned = std::max(tuned, last.last_tuned);
        const uint64_t base = b - wave.size();
        for (size_t q = 0; q < wave.size(); ++q) {
            sj_status js = st != SJ_OK ? st : wave[q].st;
            if (wave[q].path == 2) ++reruns;
            if (js == SJ_OK) {
                out[base + q] = wave[q].res;
                pairs += wave[q].res->count;
                evals += wave[q].evaluations;
                rechecks += wave[q].rechecks;
            } else if (wave[q].res) {
                sj_result_free(wave[q].res);
            }
            if (status) status[base + q] = js;
            if (js != SJ_OK && first == SJ_OK) {
                first = js;
                first_msg = st != SJ_OK ? err.msg : wave[q].msg;
            }
        }
        if (st != SJ_OK) {
            for (uint64_t i = b; i < n_jobs; ++i)
                if (status) status[i] = st;
            break;
        }
    }
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.frame = -1;   // each job chooses its own frame
    ctx->stats.pairs = pairs;
    ctx->stats.evaluations = evals;
    ctx->stats.rechecks = rechecks;
    ctx->stats.batches = (uint32_t)waves;
    ctx->stats.retries = (uint32_t)reruns;
    ctx->stats.ms_total = now_ms() - t0;
    ctx->stats.kernel_launches = launches_so_far() - l0;
    // the multi-join launch parameters of the last wave; tuned: the most
    // any wave of the call saw (2 when one was tuned)
    ctx->stats.tuned = tuned;
    ctx->stats.grab = last.last_grab;
    ctx->stats.nbuf = last.last_nbuf;
    ctx->stats.staging = last.last_eb;
    ctx->last_err = first == SJ_OK ? std::string() : first_msg;
    return first;
}

}  // extern "C"
