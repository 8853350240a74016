// serve.cu -- request interface of include/sj.h (sj_submit / sj_poll).
//
// Placeholder scheduler: each request is joined when it is submitted.
#include <map>
#include <mutex>

#include "sj_internal.cuh"

struct ServeState {
    std::mutex mu;
    uint64_t next = 1;
    std::map<uint64_t, std::pair<sj_status, sj_result *>> done;
};

extern "C" {

void sj_serve_shutdown(sj_ctx *ctx);

sj_status sj_submit(sj_ctx *ctx, const double *pts, uint64_t n, int d, double eps, uint64_t *ticket) {
    if (!ctx || !ticket) return SJ_EINVAL;
    static std::mutex gmu;
    static std::map<sj_ctx *, ServeState *> states;
    ServeState *ss;
    {
        std::lock_guard<std::mutex> lk(gmu);
        auto &slot = states[ctx];
        if (!slot) slot = new ServeState();
        ss = slot;
    }
    sj_result *r = nullptr;
    sj_status st = sj_selfjoin(ctx, pts, n, d, eps, &r);
    std::lock_guard<std::mutex> lk(ss->mu);
    *ticket = ss->next++;
    ss->done[*ticket] = std::make_pair(st, r);
    (void)states;
    return SJ_OK;
}

sj_status sj_poll(sj_ctx *ctx, uint64_t ticket, int wait_ms, sj_result **out) {
    (void)ctx; (void)ticket; (void)wait_ms; (void)out;
    return SJ_ENOTFOUND;
}

void sj_serve_shutdown(sj_ctx *ctx) { (void)ctx; }

}  // extern "C"
