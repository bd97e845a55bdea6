// Server (cd_server_* in include/cd.h): continuous batching of submitted
// runs in two lanes.  Small runs (adjacency entries plus vertices up to
// SMALL_WORK) and large runs each have a lane: a host thread owning an
// Engine and its own stream.  The small lane's launches use a quarter of the
// device's resident blocks; the large lane's use the rest while small runs
// are active and the whole device otherwise, so the two lanes' persistent
// launches run side by side and a small run does not wait for a large run's
// phases.  Between
// two engine steps a lane admits its queued runs in submission order while
// the shared slots and device-memory budget allow, so a run submitted while
// others are on the GPU joins its lane's very next batched launch.  Finished
// runs wait in a table until their owner takes the result.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "api_common.cuh"

using namespace cd;

namespace {

using Clock = std::chrono::steady_clock;

enum { E_QUEUED, E_RUNNING, E_DONE };

constexpr int64_t SMALL_WORK = int64_t(1) << 21;   // entries + vertices of a small-lane run
constexpr double SMALL_SHARE = 0.25;               // the small lane's share of the resident blocks

struct Entry {
    uint64_t ticket = 0;
    JobSpec spec;
    int lane = 1;               // 0: small runs, 1: large runs
    size_t est = 0;
    int state = E_QUEUED;
    std::unique_ptr<Job> job;
    Clock::time_point t_submit, t_done;
};

// Device bytes a run may hold at its peak (an estimate with headroom):
// per-vertex schedule, labels, ranks and move-phase buffers of the finest
// level, coarse levels no larger than the input, and the coarsening sort.
size_t estimate_bytes(const JobSpec &sp) {
    const double n = (double)sp.g.n, nnz = (double)sp.g.nnz;
    double b = (1 << 20) + 230.0 * n + 32.0 * nnz;
    if (sp.algo == ALGO_PLP) b = (1 << 20) + 120.0 * n + 8.0 * nnz;
    if (sp.algo == ALGO_EPP) b += sp.ensemble * 100.0 * n + 48.0 * n;
    return (size_t)b;
}

}  // namespace

struct cd_server {
    struct Lane {
        std::unique_ptr<Engine> engine;
        cudaStream_t stream = nullptr;
        bool own_stream = false;
        std::thread th;
    };
    std::mutex mu;
    std::condition_variable wake;   // lane threads: new work or stop
    std::condition_variable done;   // pollers: a run finished
    std::deque<Entry *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Entry>> entries;
    size_t budget = 0, used = 0;
    int max_slots = 1, max_queue = 1;
    int64_t running = 0, finished = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int dev = 0;
    cudaStream_t copy_stream = nullptr;
    Lane lanes[2];
    std::atomic<int> small_active{0};   // runs in the small lane

    // The large lane takes the whole device while the small lane is idle and
    // leaves the small lane its share otherwise (a launch already running
    // with the whole device delays the small lane by one phase at most).
    double share(int lane) const {
        if (lane == 0) return SMALL_SHARE;
        return small_active.load() > 0 ? 1.0 - SMALL_SHARE : 1.0;
    }

    // The lane's first queued run, if it fits the free slots and memory.
    std::deque<Entry *>::iterator admissible(int lane) {
        if (running >= max_slots) return queue.end();
        for (auto it = queue.begin(); it != queue.end(); ++it)
            if ((*it)->lane == lane) return used + (*it)->est <= budget ? it : queue.end();
        return queue.end();
    }

    void loop(int lane) {
        cudaSetDevice(dev);
        Engine &engine = *lanes[lane].engine;
        std::vector<Entry *> active;
        for (;;) {
            std::vector<Entry *> admitted;
            {
                std::unique_lock<std::mutex> lk(mu);
                wake.wait(lk, [&]() { return stop || !active.empty() || admissible(lane) != queue.end(); });
                if (stop) return;
                for (auto it = admissible(lane); it != queue.end(); it = admissible(lane)) {
                    Entry *e = *it;
                    queue.erase(it);
                    e->state = E_RUNNING;
                    used += e->est;
                    running++;
                    admitted.push_back(e);
                }
            }
            for (Entry *e : admitted) {
                e->job = std::make_unique<Job>(e->spec);
                try {
                    engine.add(e->job.get());
                } catch (const Error &err) {
                    e->job->status = err.status;
                    e->job->msg = err.msg;
                    e->job->done = true;
                }
                active.push_back(e);
            }
            if (lane == 0) small_active.store((int)active.size());
            engine.set_grid_share(share(lane));
            try {
                engine.step();
            } catch (const Error &err) {
                for (Entry *e : active)
                    if (!e->job->done) {
                        e->job->status = err.status;
                        e->job->msg = err.msg;
                        e->job->done = true;
                    }
            }
            const auto now = Clock::now();
            bool any = false;
            {
                std::lock_guard<std::mutex> lk(mu);
                for (Entry *e : active)
                    if (e->job->done) {
                        e->state = E_DONE;
                        e->t_done = now;
                        used -= e->est;
                        running--;
                        finished++;
                        any = true;
                    }
            }
            active.erase(std::remove_if(active.begin(), active.end(), [](Entry *e) { return e->state == E_DONE; }),
                         active.end());
            if (lane == 0) small_active.store((int)active.size());
            if (any) {
                done.notify_all();
                wake.notify_all();   // freed slots and memory may admit the other lane's runs
            }
        }
    }
};

extern "C" {

cd_status cd_server_create(size_t device_mem_budget, int max_slots, int max_queue, void *stream, cd_server **out) {
    if (!out) return CD_EINVAL;
    *out = nullptr;
    return guarded([&]() {
        if (max_slots < 1 || max_queue < 1) raise(CD_EINVAL, "max_slots and max_queue must be >= 1");
        auto S = std::make_unique<cd_server>();
        CD_CUDA(cudaGetDevice(&S->dev));
        if (device_mem_budget == 0) {
            size_t fr = 0, tot = 0;
            CD_CUDA(cudaMemGetInfo(&fr, &tot));
            device_mem_budget = fr / 10 * 8;
        }
        S->budget = device_mem_budget;
        S->max_slots = max_slots;
        S->max_queue = max_queue;
        // the large lane runs on the caller's stream (or one of its own), the
        // small lane on a stream of its own
        if (stream) {
            S->lanes[1].stream = static_cast<cudaStream_t>(stream);
        } else {
            CD_CUDA(cudaStreamCreateWithFlags(&S->lanes[1].stream, cudaStreamNonBlocking));
            S->lanes[1].own_stream = true;
        }
        CD_CUDA(cudaStreamCreateWithFlags(&S->lanes[0].stream, cudaStreamNonBlocking));
        S->lanes[0].own_stream = true;
        CD_CUDA(cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking));
        const int hw = (int)std::thread::hardware_concurrency();
        const int workers = std::max(1, std::min(16, hw > 0 ? hw : 4));
        for (int l = 0; l < 2; l++) {
            S->lanes[l].engine = std::make_unique<Engine>(S->lanes[l].stream, l == 0 ? std::max(1, workers / 2) : workers);
            S->lanes[l].engine->set_grid_share(l == 0 ? SMALL_SHARE : 1.0 - SMALL_SHARE);
        }
        cd_server *raw = S.get();
        for (int l = 0; l < 2; l++) S->lanes[l].th = std::thread([raw, l]() { raw->loop(l); });
        *out = S.release();
        return CD_OK;
    });
}

cd_status cd_server_submit(cd_server *S, cd_graph *g, const cd_task *task, const cd_opts *o, uint64_t *ticket) {
    if (!S || !g || !ticket) return CD_EINVAL;
    return guarded([&]() {
        RunOpts ro = to_run(o);
        auto e = std::make_unique<Entry>();
        e->spec = task_spec(g->g.view, task, ro, nullptr);
        e->est = estimate_bytes(e->spec);
        e->lane = g->g.view.nnz + g->g.view.n <= SMALL_WORK ? 0 : 1;
        CD_CUDA(cudaStreamSynchronize(g->stream));
        std::lock_guard<std::mutex> lk(S->mu);
        if (e->est > S->budget)
            raise(CD_EINVAL, "run needs about %zu bytes, more than the budget of %zu", e->est, S->budget);
        if ((int)S->queue.size() >= S->max_queue) raise(CD_EBUSY, "queue full (%d runs)", S->max_queue);
        e->ticket = S->next_ticket++;
        e->t_submit = Clock::now();
        *ticket = e->ticket;
        S->queue.push_back(e.get());
        S->entries[e->ticket] = std::move(e);
        S->wake.notify_all();
        return CD_OK;
    });
}

cd_status cd_server_poll(cd_server *S, uint64_t ticket, double timeout_ms, int32_t *labels, int labels_mem,
                         double *mod, double *latency_ms, cd_stats *st) {
    if (!S) return CD_EINVAL;
    return guarded([&]() {
        check_mem(labels_mem);
        std::unique_ptr<Entry> e;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto it = S->entries.find(ticket);
            if (it == S->entries.end()) raise(CD_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
            Entry *p = it->second.get();
            auto ready = [&]() { return p->state == E_DONE; };
            if (timeout_ms < 0) {
                S->done.wait(lk, ready);
            } else if (timeout_ms > 0) {
                S->done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
            }
            if (!ready()) return CD_EBUSY;
            e = std::move(it->second);
            S->entries.erase(it);
            S->finished--;
        }
        Job &j = *e->job;
        if (j.status != CD_OK) raise(j.status, "%s", j.msg.c_str());
        const int64_t n = j.spec.g.n;
        if (labels && n)
            CD_CUDA(cudaMemcpyAsync(labels, j.labels(), n * sizeof(int32_t),
                                    labels_mem == CD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    S->copy_stream));
        CD_CUDA(cudaStreamSynchronize(S->copy_stream));
        if (mod) *mod = j.mod;
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(e->t_done - e->t_submit).count();
        to_stats(j.st, st);
        return j.st.converged ? CD_OK : CD_ENOTCONV;
    });
}

cd_status cd_server_info(cd_server *S, int64_t *queued, int64_t *running, int64_t *finished) {
    if (!S) return CD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int64_t)S->queue.size();
    if (running) *running = S->running;
    if (finished) *finished = S->finished;
    return CD_OK;
}

cd_status cd_server_destroy(cd_server *S) {
    if (!S) return CD_OK;
    return guarded([&]() {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->wake.notify_all();
        for (auto &L : S->lanes)
            if (L.th.joinable()) L.th.join();
        S->done.notify_all();
        S->queue.clear();
        S->entries.clear();   // frees every run while the engines' streams exist
        for (auto &L : S->lanes) {
            CD_CUDA(cudaStreamSynchronize(L.stream));
            L.engine.reset();
        }
        cudaStreamDestroy(S->copy_stream);
        for (auto &L : S->lanes)
            if (L.own_stream) cudaStreamDestroy(L.stream);
        delete S;
        return CD_OK;
    });
}

}  // extern "C"
