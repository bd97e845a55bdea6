// Host engine (engine.cu): jobs that run PLP (Algorithm 1), PLM / PLMR
// (Algorithms 3, 4) or EPP (Algorithm 5) on one graph each.  A job advances
// through its stages on a host worker thread (colouring, schedule,
// coarsening, prolongation, compaction) until it needs a persistent phase
// (a PLM move phase or a PLP run); every phase pending at that point joins
// one batched launch, after which the jobs advance again.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "move_kernels.cuh"

namespace cd {

struct RunStats {
    int32_t levels = 0, colors0 = -1, converged = 1, ncomm = 0;
    int64_t sweeps = 0, moves = 0, iters = 0, entries = 0, candidates = 0, decisions = 0;
    double ms_color = 0, ms_move = 0, ms_coarsen = 0, ms_total = 0;
    int64_t k_launches = 0;
    double k_ms = 0, k_bytes = 0;
    double stage_ms[3] = {0, 0, 0};   // move kernel (profile mode): class steps, re-check sort, re-check
};

struct RunOpts {
    uint64_t seed = 1;
    int32_t max_sweeps = 256, max_levels = 64, max_iters = 1000;
    bool profile = false;
    bool trace = false;          // profile level 2: per-class times of the move phases
    int64_t res_p = 1, res_q = 1;   // PLM resolution gamma = res_p / res_q (reduced)
    int32_t racy = 0;            // > 0: the racy schedule with this many hash rounds per sweep (not deterministic)
    int64_t scratch_budget = 0;  // > 0: low-memory mode, bytes of coarsening scratch per pass
    int32_t int_path = 0;        // gain width: 0 the narrowest exact one, 64, or 128
    int64_t team_quantum = int64_t(1) << 18;   // launch shape (speed only)
    int32_t team_min = 8;
    BinLimits bins{{4, 16, 128, BLK_MAXDEG, BLK_MAXDEG}};  // schedule degree bins (speed only)
};

enum Algo { ALGO_PLP = 0, ALGO_PLM = 1, ALGO_EPP = 2 };

struct JobSpec {
    GraphView g;
    int algo = ALGO_PLM;
    bool refine = false;        // PLM: PLMR; EPP: refinement in the final PLM
    int ensemble = 1;           // EPP: number of PLP base runs
    double theta = 0;           // PLP / EPP bases: stop once at most theta labels change
    RunOpts o;
    int32_t *labels = nullptr;  // device, g.n entries; nullptr: the job keeps its own
    bool want_mod = false;      // compute the modularity of the result
};

struct JobState;

// A job's kernels, copies and stream-ordered allocations all go to one
// stream for the job's whole life, whichever host thread advances it, so a
// buffer freed by the job is never reused while the job's own earlier work
// on it is still queued.
struct Job {
    JobSpec spec;
    RunStats st;
    cd_status status = CD_OK;   // CD_OK until a step fails
    std::string msg;
    int64_t fail_order = -1;    // order of the failure among all jobs (earliest first)
    bool done = false;
    double mod = 0;
    DBuf<int32_t> own_labels;   // used when spec.labels is nullptr
    std::unique_ptr<JobState> state;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    explicit Job(const JobSpec &s);
    ~Job();
    void release();             // frees the job's working memory and stream
    int32_t *labels() const { return spec.labels ? spec.labels : own_labels.p; }
};

struct PhaseRun;
class WorkerPool;


class Engine {
  public:
    // Batched launches run on `s`; `workers` host threads (0: the caller's
    // thread, on `s`) advance the jobs.
    Engine(cudaStream_t s, int workers);
    ~Engine();
    Engine(const Engine &) = delete;
    Engine &operator=(const Engine &) = delete;
    void add(Job *j);            // the caller keeps ownership; j stays valid until done
    void step();                 // advances every unfinished job through one phase
    // Fraction (0, 1] of the device's resident blocks that this engine's
    // launches use, so that engines with shares summing to at most 1 run
    // their persistent launches side by side.
    void set_grid_share(double share) { share_ = share; }
    bool busy() const { return !active_.empty(); }
    size_t active() const { return active_.size(); }
    int64_t launches = 0;        // batched launches so far

  private:
    void launch(std::vector<PhaseRun *> &runs);
    void ensure_block_tables(int blocks);
    cudaStream_t s_;
    double share_ = 1.0;
    DBuf<int32_t> gt_keys_;            // role-3b tables of the launches
    DBuf<unsigned long long> gt_vals_;
    int gt_blocks_ = 0;
    std::unique_ptr<WorkerPool> pool_;
    std::vector<Job *> active_;
};

// Runs the jobs to completion; the earliest failure is raised after every
// job has stopped.
void run_jobs(std::vector<Job *> &jobs, cudaStream_t s, int workers);

// The batch engine's launch planner on bare phase sizes (host only): tiers
// of teams over a grid of at most `grid_max` blocks, and the order in which
// the runs are placed into the tiers.
struct PlanTier {
    int32_t begin, blocks;      // block range [begin, begin + blocks)
    int32_t team_size, team0;   // blocks per team; index of the tier's first team
    int32_t first, count;       // runs [first, first + count) of `order`
};
struct PlanView {
    int32_t grid = 0, nteams = 0;
    std::vector<PlanTier> tiers;
    std::vector<int32_t> order;
};
PlanView plan_for_sizes(const std::vector<int64_t> &work, int64_t quantum, int32_t team_min, int grid_max);

// Single-graph drivers (one job on the caller's thread).  Labels are written
// to `labels` (device, g.n entries), compacted.
void run_plm(const GraphView &g, bool refine, const RunOpts &o, int32_t *labels, RunStats &st, cudaStream_t s);
void run_plp(const GraphView &g, const RunOpts &o, double theta, int32_t *labels, RunStats &st, cudaStream_t s);
void run_epp(const GraphView &g, int b, bool final_refine, const RunOpts &o, double theta, int32_t *labels,
             RunStats &st, cudaStream_t s);
// EPP(b, Base, Final) with up to `rounds` ensemble rounds (cd_epp_general).
enum { EPP_BASE_PLP = 0, EPP_BASE_PLM = 1, EPP_BASE_PLMR = 2 };
void run_epp_general(const GraphView &g, int b, int base, bool final_refine, int rounds, const RunOpts &o,
                     double theta, int32_t *labels, RunStats &st, cudaStream_t s);

// Class trace of the move phases run with RunOpts::trace (profile level 2):
// TRACE_FIELDS int64 per class step, appended in completion order.
// phase, sweep, class, vertices, entries, hub chunks, hub slices, hubs >
// HUB_RELAX, ns, then the latest end of the items, the hub-decide slices and
// the finisher's work and the latest start of a block's first item, in ns
// from the class start (0: stage absent), the longest lane-group, block and
// hub-chunk item, decide-slice wait and decide slice (ns), and the class's
// applied moves (early sweeps) or re-check candidates (late sweeps)
constexpr int TRACE_FIELDS = 19;
std::vector<int64_t> take_class_trace();

}  // namespace cd
