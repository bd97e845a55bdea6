// Launch-shape autotuner (cd_tune in include/cd.h).
//
// The options it tunes change how work is laid out on the GPU but never a
// result: team_quantum and team_min shape the tiers and teams of shared
// launches, and bin_max moves vertices between the 4-lane, 8-lane, warp,
// block and hub roles (vertices of a colour class decide independently of
// one another, so the role a vertex gets cannot change its decision).  The
// tuner therefore measures complete runs of the caller's own task and keeps
// whichever shape is fastest: coordinate descent over one option at a time,
// a candidate replacing the current shape only when it is at least 1% faster.
#include <algorithm>
#include <chrono>
#include <memory>
#include <thread>
#include <vector>

#include "api_common.cuh"

using namespace cd;

namespace {

double timed_run(const std::vector<cd_graph *> &gs, const cd_task *task, const cd_opts &o, cudaStream_t s,
                 int workers) {
    const RunOpts ro = to_run(&o);
    std::vector<std::unique_ptr<Job>> jobs;
    std::vector<Job *> jp;
    for (cd_graph *g : gs) {
        JobSpec sp = task_spec(g->g.view, task, ro, nullptr);
        sp.want_mod = false;
        jobs.push_back(std::make_unique<Job>(sp));
        jp.push_back(jobs.back().get());
    }
    CD_CUDA(cudaStreamSynchronize(s));
    const auto t0 = std::chrono::steady_clock::now();
    run_jobs(jp, s, workers);
    CD_CUDA(cudaStreamSynchronize(s));
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" cd_status cd_tune(cd_graph *const *gs, int count, const cd_task *task, const cd_opts *base,
                             int max_trials, cd_opts *best, double *best_ms, void *stream) {
    if (!best) return CD_EINVAL;
    return guarded([&]() {
        if (count < 1 || !gs) raise(CD_EINVAL, "count must be >= 1 and gs non-NULL");
        if (max_trials < 1) raise(CD_EINVAL, "max_trials must be >= 1");
        std::vector<cd_graph *> v;
        for (int i = 0; i < count; i++) {
            if (!gs[i]) raise(CD_EINVAL, "graph %d is NULL", i);
            CD_CUDA(cudaStreamSynchronize(gs[i]->stream));
            v.push_back(gs[i]);
        }
        cd_opts cur;
        cd_opts_default(&cur);
        if (base) cur = *base;
        for (int i = 0; i < NLIM; i++)
            if (cur.bin_max[i] == 0) cur.bin_max[i] = BIN_DEFAULT[i];
        to_run(&cur);   // validates the base options
        (void)task_spec(v[0]->g.view, task, to_run(&cur), nullptr);   // validates the task
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int hw = (int)std::thread::hardware_concurrency();
        const int workers = count > 1 ? std::max(1, std::min({16, count, hw > 0 ? hw : 4})) : 0;

        double cur_ms = timed_run(v, task, cur, s, workers);
        int trials = 1;
        // candidate values, one option at a time
        struct Axis {
            int which;                      // 0 quantum, 1 team_min, 2..6 bin_max[0..4]
            std::vector<int64_t> values;
        };
        std::vector<Axis> axes;
        const bool shared = count > 1 || task->algo == CD_ALGO_EPP;   // team shape matters
        if (shared) {
            axes.push_back({0, {int64_t(1) << 14, int64_t(1) << 16, int64_t(1) << 18, int64_t(1) << 20,
                                int64_t(1) << 22}});
            axes.push_back({1, {1, 2, 4, 8, 16, 32}});
        }
        axes.push_back({6, {1024, 2048, 4096}});
        axes.push_back({5, {256, 512, 1024}});
        axes.push_back({4, {32, 64, 128}});
        axes.push_back({3, {8, 12, 16}});
        axes.push_back({2, {2, 3, 4}});
        for (const Axis &ax : axes) {
            for (int64_t val : ax.values) {
                if (trials >= max_trials) break;
                cd_opts o = cur;
                if (ax.which == 0) {
                    if (o.team_quantum == val) continue;
                    o.team_quantum = val;
                } else if (ax.which == 1) {
                    if (o.team_min == (int32_t)val) continue;
                    o.team_min = (int32_t)val;
                } else {
                    const int b = ax.which - 2;
                    if (o.bin_max[b] == (int32_t)val) continue;
                    o.bin_max[b] = (int32_t)val;
                    bool ok = true;
                    for (int i = 1; i < NLIM; i++) ok = ok && o.bin_max[i] >= o.bin_max[i - 1];
                    if (!ok) continue;
                }
                const double ms = timed_run(v, task, o, s, workers);
                trials++;
                if (ms < 0.99 * cur_ms) {
                    cur = o;
                    cur_ms = ms;
                }
            }
        }
        *best = cur;
        if (best_ms) *best_ms = cur_ms;
        return CD_OK;
    });
}
