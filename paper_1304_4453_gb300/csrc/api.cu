// C ABI (include/cd.h): argument checks, host/device staging of caller
// buffers, error translation.  All computation happens in the engine.
#include <algorithm>
#include <memory>
#include <new>
#include <thread>

#include "common.cuh"
#include "engine.cuh"
#include "graph.cuh"

#include "api_common.cuh"

using namespace cd;

namespace {

// Device view of caller labels (copied in when they live on the host).
struct LabelsIn {
    DBuf<int32_t> tmp;
    const int32_t *p = nullptr;
    LabelsIn(const int32_t *labels, int mem, int64_t n, cudaStream_t s) {
        check_mem(mem);
        if (n > 0 && !labels) raise(CD_EINVAL, "labels is NULL");
        if (mem == CD_MEM_DEVICE) { p = labels; return; }
        tmp.alloc(n, s);
        if (n) CD_CUDA(cudaMemcpyAsync(tmp.p, labels, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        p = tmp.p;
    }
};

// Device buffer for results, copied out to host memory when needed.
struct LabelsOut {
    DBuf<int32_t> tmp;
    int32_t *dst, *p;
    int mem;
    int64_t n;
    cudaStream_t s;
    LabelsOut(int32_t *labels, int mem_, int64_t n_, cudaStream_t s_) : dst(labels), mem(mem_), n(n_), s(s_) {
        check_mem(mem);
        if (n > 0 && !labels) raise(CD_EINVAL, "labels is NULL");
        if (mem == CD_MEM_DEVICE) { p = labels; return; }
        tmp.alloc(n, s);
        p = tmp.p;
    }
    void finish() {
        if (mem == CD_MEM_HOST && n)
            CD_CUDA(cudaMemcpyAsync(dst, p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
    }
};

cd_status finish_run(const RunStats &r, cd_stats *st) {
    to_stats(r, st);
    return r.converged ? CD_OK : CD_ENOTCONV;
}

}  // namespace

extern "C" {

void cd_opts_default(cd_opts *o) {
    if (!o) return;
    o->seed = 1;
    o->max_sweeps = 256;
    o->max_levels = 64;
    o->max_iters = 1000;
    o->profile = 0;
    o->team_quantum = int64_t(1) << 18;
    o->team_min = 8;
    o->reserved = 0;
    for (int i = 0; i < NLIM; i++) o->bin_max[i] = BIN_DEFAULT[i];
    o->res_num = 1;
    o->res_den = 1;
    o->schedule = 0;
    o->int_path = 0;
    o->scratch_budget = 0;
}

const char *cd_status_str(cd_status s) {
    switch (s) {
        case CD_OK: return "CD_OK";
        case CD_EINVAL: return "CD_EINVAL";
        case CD_ENOMEM: return "CD_ENOMEM";
        case CD_ECUDA: return "CD_ECUDA";
        case CD_ENOTCONV: return "CD_ENOTCONV";
        case CD_EBUSY: return "CD_EBUSY";
        case CD_ETIMEOUT: return "CD_ETIMEOUT";
    }
    return "CD_UNKNOWN";
}

const char *cd_last_error(void) { return cd::last_error().c_str(); }

cd_status cd_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w, int mem_flags,
                          void *stream, cd_graph **out) {
    if (!out) return CD_EINVAL;
    *out = nullptr;
    return guarded([&]() {
        auto *g = new cd_graph();
        g->stream = static_cast<cudaStream_t>(stream);
        try {
            build_graph(n, row_ptr, col, w, mem_flags, g->stream, g->g);
        } catch (...) {
            cudaStream_t st = g->stream;
            delete g;
            cudaStreamSynchronize(st);
            throw;
        }
        g->m = g->g.view.nnz / 2;
        *out = g;
        return CD_OK;
    });
}

cd_status cd_graph_destroy(cd_graph *g) {
    if (!g) return CD_OK;
    return guarded([&]() {
        cudaStream_t s = g->stream;
        delete g;
        CD_CUDA(cudaStreamSynchronize(s));
        return CD_OK;
    });
}

cd_status cd_graph_info(const cd_graph *g, int64_t *n, int64_t *m, int64_t *total_weight) {
    if (!g) return CD_EINVAL;
    if (n) *n = g->g.view.n;
    if (m) *m = g->m;
    if (total_weight) *total_weight = g->g.view.W;
    return CD_OK;
}

cd_status cd_modularity(cd_graph *g, const int32_t *labels, int labels_mem, double *mod) {
    if (!g || !mod) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        LabelsIn in(labels, labels_mem, v.n, g->stream);
        if (!labels_in_range(in.p, v.n, g->stream)) raise(CD_EINVAL, "label out of range [0, n)");
        *mod = modularity(v, in.p, g->stream);
        return CD_OK;
    });
}

cd_status cd_plp(cd_graph *g, const cd_opts *o, double theta, int32_t *labels, int labels_mem, double *mod,
                 cd_stats *st) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        RunOpts ro = to_run(o);
        if (theta < 0) theta = (double)v.n * 1e-5;
        LabelsOut out(labels, labels_mem, v.n, g->stream);
        RunStats r;
        run_plp(v, ro, theta, out.p, r, g->stream);
        if (mod) *mod = modularity(v, out.p, g->stream);
        out.finish();
        return finish_run(r, st);
    });
}

cd_status cd_plm(cd_graph *g, int refine, const cd_opts *o, int32_t *labels, int labels_mem, double *mod,
                 cd_stats *st) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        if (refine != 0 && refine != 1) raise(CD_EINVAL, "refine must be 0 or 1");
        RunOpts ro = to_run(o);
        LabelsOut out(labels, labels_mem, v.n, g->stream);
        RunStats r;
        run_plm(v, refine == 1, ro, out.p, r, g->stream);
        if (mod) *mod = modularity(v, out.p, g->stream);
        out.finish();
        return finish_run(r, st);
    });
}

cd_status cd_epp(cd_graph *g, int ensemble_size, int final_refine, const cd_opts *o, int32_t *labels,
                 int labels_mem, double *mod, cd_stats *st) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        if (ensemble_size < 1) raise(CD_EINVAL, "ensemble_size must be >= 1");
        if (final_refine != 0 && final_refine != 1) raise(CD_EINVAL, "final_refine must be 0 or 1");
        RunOpts ro = to_run(o);
        LabelsOut out(labels, labels_mem, v.n, g->stream);
        RunStats r;
        run_epp(v, ensemble_size, final_refine == 1, ro, (double)v.n * 1e-5, out.p, r, g->stream);
        if (mod) *mod = modularity(v, out.p, g->stream);
        out.finish();
        return finish_run(r, st);
    });
}

cd_status cd_epp_general(cd_graph *g, int ensemble_size, int base, int final_refine, int rounds, const cd_opts *o,
                         int32_t *labels, int labels_mem, double *mod, cd_stats *st) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        if (ensemble_size < 1) raise(CD_EINVAL, "ensemble_size must be >= 1");
        if (base < CD_BASE_PLP || base > CD_BASE_PLMR) raise(CD_EINVAL, "base must be CD_BASE_PLP, _PLM or _PLMR");
        if (final_refine != 0 && final_refine != 1) raise(CD_EINVAL, "final_refine must be 0 or 1");
        if (rounds < 1 || rounds > 64) raise(CD_EINVAL, "rounds must be in [1, 64]");
        RunOpts ro = to_run(o);
        LabelsOut out(labels, labels_mem, v.n, g->stream);
        RunStats r;
        run_epp_general(v, ensemble_size, base, final_refine == 1, rounds, ro, (double)v.n * 1e-5, out.p, r,
                        g->stream);
        if (mod) *mod = modularity(v, out.p, g->stream);
        out.finish();
        return finish_run(r, st);
    });
}

cd_status cd_run_batch(cd_graph *const *gs, int count, const cd_task *task, const cd_opts *o,
                       int32_t *const *labels, int labels_mem, double *mods, cd_stats *st, void *stream) {
    return guarded([&]() {
        if (count < 0) raise(CD_EINVAL, "count must be >= 0");
        if (count > 0 && (!gs || !labels)) raise(CD_EINVAL, "gs and labels are required");
        check_mem(labels_mem);
        RunOpts ro = to_run(o);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        std::vector<std::unique_ptr<Job>> jobs;
        std::vector<Job *> jp;
        for (int i = 0; i < count; i++) {
            if (!gs[i]) raise(CD_EINVAL, "graph %d is NULL", i);
            const GraphView &v = gs[i]->g.view;
            if (v.n > 0 && !labels[i]) raise(CD_EINVAL, "labels[%d] is NULL", i);
            CD_CUDA(cudaStreamSynchronize(gs[i]->stream));
            jobs.push_back(std::make_unique<Job>(
                task_spec(v, task, ro, labels_mem == CD_MEM_DEVICE ? labels[i] : nullptr)));
            jp.push_back(jobs.back().get());
        }
        if (count == 0) return CD_OK;
        const int hw = (int)std::thread::hardware_concurrency();
        const int workers = std::max(1, std::min({16, count, hw > 0 ? hw : 4}));
        run_jobs(jp, s, workers);
        bool notconv = false;
        for (int i = 0; i < count; i++) {
            const Job &j = *jobs[i];
            if (labels_mem == CD_MEM_HOST && j.spec.g.n)
                CD_CUDA(cudaMemcpyAsync(labels[i], j.labels(), j.spec.g.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            if (mods) mods[i] = j.mod;
            if (st) to_stats(j.st, st + i);
            notconv = notconv || !j.st.converged;
        }
        CD_CUDA(cudaStreamSynchronize(s));
        return notconv ? CD_ENOTCONV : CD_OK;
    });
}

cd_status cd_plm_batch(cd_graph *const *gs, int count, int refine, const cd_opts *o, int32_t *const *labels,
                       int labels_mem, double *mods, cd_stats *st) {
    cd_task t = {CD_ALGO_PLM, refine, 1, 0, -1.0};
    void *stream = (count > 0 && gs && gs[0]) ? static_cast<void *>(gs[0]->stream) : nullptr;
    return cd_run_batch(gs, count, &t, o, labels, labels_mem, mods, st, stream);
}

cd_status cd_color(cd_graph *g, uint64_t seed, int32_t *colors, int colors_mem, int32_t *ncolors) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        LabelsOut out(colors, colors_mem, v.n, g->stream);
        int32_t k = color_graph(v, seed, out.p, g->stream);
        out.finish();
        if (ncolors) *ncolors = k;
        return CD_OK;
    });
}

cd_status cd_coarsen(cd_graph *g, const int32_t *labels, int labels_mem, cd_graph **coarse) {
    if (!g || !coarse) return CD_EINVAL;
    *coarse = nullptr;
    return guarded([&]() {
        const GraphView &v = g->g.view;
        LabelsIn in(labels, labels_mem, v.n, g->stream);
        if (!labels_in_range(in.p, v.n, g->stream)) raise(CD_EINVAL, "label out of range [0, n)");
        auto *c = new cd_graph();
        c->stream = g->stream;
        try {
            DBuf<int64_t> rank(v.n, g->stream);
            coarsen_graph(v, in.p, rank.p, c->g, g->stream);
            CD_CUDA(cudaStreamSynchronize(g->stream));
        } catch (...) {
            delete c;
            throw;
        }
        c->m = c->g.view.nnz / 2;
        *coarse = c;
        return CD_OK;
    });
}

cd_status cd_graph_export(const cd_graph *g, int64_t *row_ptr, int32_t *col, int64_t *w, int mem,
                          int64_t *nnz_out) {
    if (!g) return CD_EINVAL;
    return guarded([&]() {
        check_mem(mem);
        int64_t nnz = export_graph(g->g.view, row_ptr, col, w, mem, g->stream);
        if (nnz_out) *nnz_out = nnz;
        return CD_OK;
    });
}

void cd_debug_fail_alloc(int k) { set_alloc_failure(k); }

cd_status cd_debug_plan_launch(const int64_t *work, int count, int64_t team_quantum, int32_t team_min, int grid_max,
                               int32_t *grid, int32_t *ntiers, int32_t *tiers, int32_t *order) {
    if (!work || !grid || !ntiers || !tiers || !order) return CD_EINVAL;
    return guarded([&]() {
        if (count < 1 || team_quantum < 1 || team_min < 1 || grid_max < 1)
            raise(CD_EINVAL, "count, team_quantum, team_min and grid_max must be >= 1");
        const PlanView v = plan_for_sizes(std::vector<int64_t>(work, work + count), team_quantum, team_min, grid_max);
        *grid = v.grid;
        *ntiers = (int32_t)v.tiers.size();
        for (size_t i = 0; i < v.tiers.size(); i++) {
            const PlanTier &t = v.tiers[i];
            const int32_t row[6] = {t.begin, t.blocks, t.team_size, t.team0, t.first, t.count};
            for (int k = 0; k < 6; k++) tiers[6 * i + k] = row[k];
        }
        for (int i = 0; i < count; i++) order[i] = v.order[i];
        return CD_OK;
    });
}

cd_status cd_debug_class_trace(int64_t *out, int64_t cap, int64_t *count) {
    if (!count) return CD_EINVAL;
    return guarded([&]() {
        static std::vector<int64_t> pending;
        if (pending.empty()) pending = take_class_trace();
        const int64_t rows = (int64_t)pending.size() / TRACE_FIELDS;
        *count = rows;
        if (!out) return CD_OK;
        if (cap < rows) raise(CD_EINVAL, "class trace holds %lld rows, buffer %lld", (long long)rows, (long long)cap);
        std::copy(pending.begin(), pending.end(), out);
        pending.clear();
        return CD_OK;
    });
}

uint64_t cd_launch_count(void) { return launch_count(); }

cd_status cd_memory_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, int reset_high) {
    return guarded([&]() {
        pool_stats(used, used_high, reserved, reset_high != 0);
        return CD_OK;
    });
}

}  // extern "C"
