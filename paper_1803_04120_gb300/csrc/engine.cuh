// engine.cuh -- the multi-join engine (engine.cu): many self-joins per pass,
// used by sj_selfjoin_multi and by the serving scheduler of sj_submit.
#pragma once

#include <string>
#include <vector>

#include "sj_internal.cuh"

namespace sj {

// One join of a wave, as the caller describes it and as the engine returns it.
struct EngJob {
    const void *pts = nullptr;   // n x d FP64, host (pinned or pageable) or device memory
    uint64_t n = 0;
    int d = 0;
    double eps = 0;
    // results
    sj_status st = SJ_OK;
    std::string msg;
    sj_result *res = nullptr;    // host result, owned by the caller afterwards
    uint64_t evaluations = 0, rechecks = 0;
    int path = 0;                // 0 multi-join launch, 1 stand-alone join, 2 rerun after overflow
};

// Counters of an engine since it was created.
struct EngStats {
    uint64_t waves = 0, jobs = 0, graph_launches = 0, kernel_nodes = 0;
    uint64_t overflow_reruns = 0, standalone = 0;
    uint64_t tuned_waves = 0;    // waves whose multi-join launch was tuned
    double ms_tune = 0;          // host wall time of those tuning passes
    // the last wave's launch: 0 defaults (or forced), 1 the wave tuner's
    // cached choice, 2 tuned by that wave; its parameters (0: by dimension)
    int last_tuned = 0, last_grab = 1, last_nbuf = 0, last_eb = 0, last_slots = 0;
    double ms_bounds = 0, ms_graph = 0, ms_output = 0;
};

class Engine;

// Creates an engine on `device` with the configuration of a context (the
// precision, the sort flag and the launch tuning are taken from it).
sj_status engine_create(Error &err, int device, const sj_config &cfg, Engine **out);
void engine_destroy(Engine *e);
// Runs up to kMultiJobs joins: one bounds pass (one host read-back), one
// replay of the engine's CUDA graph (batched index build of every job and
// one persistent multi-join launch), then the results to pinned host memory.
// Per-job failures are reported in the job; the return value is SJ_OK unless
// the engine itself failed.  on_done (optional) is called once per job, from
// the calling thread, as soon as that job's result is on the host (or the
// job failed): smaller results first.
sj_status engine_run(Error &err, Engine *e, EngJob *const *jobs, int k,
                     void (*on_done)(void *user, int job) = nullptr, void *user = nullptr);
EngStats engine_stats(const Engine *e);
// Forgets the choices of the wave tuner (the next wave of every key is
// tuned again).
void engine_tune_reset();

// Device bytes a job is expected to hold in the engine (points, index,
// result buffer), from the bounding box of a sample of its points, and the
// expected pair count.  pts must be host memory.
uint64_t engine_estimate(const double *pts, uint64_t n, int d, double eps, uint64_t *pairs);

}  // namespace sj
