// Helpers shared by the C ABI translation units (api.cu, server.cu):
// exception-to-status translation, option and statistics conversion.
#pragma once
#include <new>

#include "common.cuh"
#include "engine.cuh"

namespace cd {

const std::string &last_error();

template <typename F>
cd_status guarded(F &&f) {
    try {
        cd_status s = f();
        if (s == CD_OK) set_last_error("");
        return s;
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return CD_ENOMEM;
    } catch (...) {
        set_last_error("unexpected internal error");
        return CD_ECUDA;
    }
}

inline RunOpts to_run(const cd_opts *o) {
    cd_opts d;
    cd_opts_default(&d);
    if (!o) o = &d;
    if (o->max_sweeps < 1 || o->max_levels < 1 || o->max_iters < 0)
        raise(CD_EINVAL, "max_sweeps and max_levels must be >= 1, max_iters >= 0");
    if (o->team_quantum < 1 || o->team_min < 1) raise(CD_EINVAL, "team_quantum and team_min must be >= 1");
    RunOpts r;
    r.seed = o->seed;
    r.max_sweeps = o->max_sweeps;
    r.max_levels = o->max_levels;
    r.max_iters = o->max_iters;
    r.profile = o->profile != 0;
    r.trace = o->profile >= 2;
    int64_t rp_ = o->res_num, rq_ = o->res_den;
    if (rp_ == 0 && rq_ == 0) rp_ = rq_ = 1;
    if (rp_ < 0 || rq_ < 1) raise(CD_EINVAL, "resolution %lld / %lld: need res_num >= 0, res_den >= 1",
                                  (long long)o->res_num, (long long)o->res_den);
    for (int64_t a = rp_, b = rq_;;) {   // reduce by the gcd (same decisions, smaller products)
        if (b == 0) {
            if (a > 1) { rp_ /= a; rq_ /= a; }
            break;
        }
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    r.res_p = rp_;
    r.res_q = rq_;
    if (o->schedule < 0 || o->schedule > 4096)
        raise(CD_EINVAL, "schedule %d: 0 (colour classes) or 1..4096 (racy rounds per sweep)", o->schedule);
    r.racy = o->schedule;
    if (o->scratch_budget < 0) raise(CD_EINVAL, "scratch_budget must be >= 0");
    r.scratch_budget = o->scratch_budget;
    if (o->int_path != 0 && o->int_path != 64 && o->int_path != 128)
        raise(CD_EINVAL, "int_path %d: 0 (automatic), 64 or 128", o->int_path);
    r.int_path = o->int_path;
    r.team_quantum = o->team_quantum;
    r.team_min = o->team_min;
    for (int i = 0; i < NLIM; i++) {
        const int32_t v = o->bin_max[i] ? o->bin_max[i] : BIN_DEFAULT[i];
        if (v < 1 || v > BIN_CAP[i] || (i > 0 && v < r.bins.lim[i - 1]))
            raise(CD_EINVAL, "bin_max[%d] = %d outside [bin_max[%d], %d]", i, v, i - 1, BIN_CAP[i]);
        r.bins.lim[i] = v;
    }
    return r;
}

inline void to_stats(const RunStats &r, cd_stats *st) {
    if (!st) return;
    st->levels = r.levels;
    st->colors0 = r.colors0 < 0 ? 0 : r.colors0;
    st->converged = r.converged;
    st->ncomm = r.ncomm;
    st->sweeps = r.sweeps;
    st->moves = r.moves;
    st->iters = r.iters;
    st->entries = r.entries;
    st->candidates = r.candidates;
    st->decisions = r.decisions;
    st->ms_color = r.ms_color;
    st->ms_move = r.ms_move;
    st->ms_coarsen = r.ms_coarsen;
    st->ms_total = r.ms_total;
    st->k_launches = r.k_launches;
    st->k_ms = r.k_ms;
    st->k_bytes = r.k_bytes;
    st->stage_items_ms = r.stage_ms[0];
    st->stage_sort_ms = r.stage_ms[1];
    st->stage_recheck_ms = r.stage_ms[2];
}

inline void check_mem(int mem) {
    if (mem != CD_MEM_HOST && mem != CD_MEM_DEVICE) raise(CD_EINVAL, "unknown memory flag %d", mem);
}

// Job of a cd_task on a graph (validated); labels nullptr: job-owned.
inline JobSpec task_spec(const GraphView &g, const cd_task *t, const RunOpts &o, int32_t *labels) {
    if (!t) raise(CD_EINVAL, "task is NULL");
    JobSpec sp;
    sp.g = g;
    sp.o = o;
    sp.labels = labels;
    sp.want_mod = true;
    if (t->refine != 0 && t->refine != 1) raise(CD_EINVAL, "refine must be 0 or 1");
    sp.refine = t->refine == 1;
    switch (t->algo) {
    case CD_ALGO_PLP:
        sp.algo = ALGO_PLP;
        sp.theta = t->theta < 0 ? (double)g.n * 1e-5 : t->theta;
        break;
    case CD_ALGO_PLM:
        sp.algo = ALGO_PLM;
        break;
    case CD_ALGO_EPP:
        if (t->ensemble < 1) raise(CD_EINVAL, "ensemble must be >= 1");
        sp.algo = ALGO_EPP;
        sp.ensemble = t->ensemble;
        sp.theta = (double)g.n * 1e-5;
        break;
    default:
        raise(CD_EINVAL, "unknown algorithm %d", t->algo);
    }
    return sp;
}

}  // namespace cd
