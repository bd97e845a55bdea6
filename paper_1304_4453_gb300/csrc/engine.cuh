// Host drivers of PLP, PLM/PLMR and EPP (engine.cu).
#pragma once
#include "common.cuh"

namespace cd {

struct RunStats {
    int32_t levels = 0, colors0 = -1, converged = 1, ncomm = 0;
    int64_t sweeps = 0, moves = 0, iters = 0, entries = 0, candidates = 0, decisions = 0;
    double ms_color = 0, ms_move = 0, ms_coarsen = 0, ms_total = 0;
    int64_t k_launches = 0;
    double k_ms = 0, k_bytes = 0;
    double stage_ms[3] = {0, 0, 0};   // move kernel: items, hub decide, re-check (profile mode)
};

struct RunOpts {
    uint64_t seed = 1;
    int32_t max_sweeps = 256, max_levels = 64, max_iters = 1000;
    bool profile = false;
};

// Labels are written to `labels` (device, g.n entries), compacted.
void run_plm(const GraphView &g, bool refine, const RunOpts &o, int32_t *labels, RunStats &st, cudaStream_t s);
void run_plp(const GraphView &g, const RunOpts &o, double theta, int32_t *labels, RunStats &st, cudaStream_t s);
void run_epp(const GraphView &g, int b, bool final_refine, const RunOpts &o, double theta, int32_t *labels,
             RunStats &st, cudaStream_t s);

}  // namespace cd
