/*
 * cd.h -- C ABI of the GB300 community-detection library (libcdgpu.so).
 *
 * Implements the parallel community-detection methods of Staudt & Meyerhenke,
 * "Engineering Parallel Algorithms for Community Detection in Massive
 * Networks": label propagation PLP (Algorithm 1), the Louvain method PLM
 * (Algorithms 2, 3), PLM with refinement PLMR (Algorithm 4) and ensemble
 * preprocessing EPP (Algorithm 5), with modularity (Eq. 1) as the quality
 * measure.  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *  - Graph (Section III, notation): undirected, n vertices with ids 0..n-1,
 *    positive integer edge weights.  Input is a symmetric CSR: row_ptr
 *    int64[n+1] with row_ptr[0] = 0, col int32[row_ptr[n]] sorted strictly
 *    ascending inside each row, (u,v,w) present iff (v,u,w) is, a self-loop
 *    {u,u} stored once in row u.  w int32[row_ptr[n]] with every w > 0, or
 *    NULL for unit weights.  n < 2^31.
 *  - A solution (Section III) is an int32 array indexed by vertex holding
 *    community ids.  Outputs are compacted: ids are 0..k-1, numbered in
 *    ascending order of the raw ids the algorithm produced.
 *  - Memory flags say where a caller pointer lives: CD_MEM_HOST (pageable or
 *    pinned host memory) or CD_MEM_DEVICE (device memory of the current CUDA
 *    device).  Output buffers are caller-owned and must hold n entries.
 *  - Every call runs on the stream given to cd_graph_create and returns only
 *    when its results are written (synchronous), except where noted.
 *  - No call aborts, traps or prints.  Failures return a cd_status; a
 *    thread-local message is available from cd_last_error().
 *  - CD_ENOTCONV: a move phase or PLP hit its iteration cap; the labels and
 *    modularity returned are still valid.
 *  - Determinism: for the same graph, options and seed, results are
 *    bit-identical from run to run and equal to the CPU oracle's.
 */
#ifndef CD_H
#define CD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cd_graph cd_graph;
typedef struct cd_server cd_server;

typedef enum {
    CD_OK = 0,
    CD_EINVAL = 1,     /* invalid argument or malformed CSR; nothing allocated */
    CD_ENOMEM = 2,     /* device or host allocation failed; nothing leaked */
    CD_ECUDA = 3,      /* a CUDA runtime call failed (see cd_last_error) */
    CD_ENOTCONV = 4,   /* iteration cap reached; results still valid */
    CD_EBUSY = 5,      /* server queue full, or a polled job is not finished */
    CD_ETIMEOUT = 6    /* a bounded wait ran out */
} cd_status;

enum { CD_MEM_HOST = 0, CD_MEM_DEVICE = 1, CD_BORROW = 2 };

/* Options.  cd_opts_default() fills: seed 1, max_sweeps 256, max_levels 64,
 * max_iters 1000, profile 0, team_quantum 262144, team_min 8,
 * bin_max {4, 16, 128, 1024, 1024} (the global-table block role is empty).
 *   seed        colouring priorities (Jones-Plassmann) and the PLP tie order
 *               derive from it; EPP base i uses seed+i.
 *   max_sweeps  cap on sweeps of one move phase (Algorithm 2 "repeat").
 *   max_levels  cap on the coarsening hierarchy depth (Algorithm 3).
 *   max_iters   cap on PLP iterations (Algorithm 1 "while").
 *   profile     1: time every persistent launch with CUDA events and report
 *               it in cd_stats (adds host synchronisation).  2: also trace
 *               every class step of the move phases (cd_debug_class_trace).
 *   team_quantum, team_min  launch shape of shared launches (EPP bases,
 *               batches, the server): a graph whose work (adjacency entries
 *               + vertices) is w gets teams of at least
 *               ceil(w / team_quantum) blocks rounded up to a power of two,
 *               and up to team_min graphs of a tier run side by side.  They
 *               change speed only, never results.
 *   bin_max     degree limits of the schedule's vertex roles: degree <=
 *               bin_max[0] -> 4 lanes, <= bin_max[1] -> 8 lanes, <= bin_max[2]
 *               -> a warp, <= bin_max[3] -> a block with a shared-memory
 *               table, <= bin_max[4] -> a block with a table in global
 *               memory, above -> multi-block hub path.  Limits may not exceed
 *               4, 16, 128, 1024, 4096 and must not decrease (0 keeps the
 *               default).  Speed only, never results.
 *   res_num, res_den  the resolution gamma = res_num / res_den of Section
 *               III-B, read as a factor on the volume term of the move gain:
 *               the moves maximise sum_C omega(C)/W - gamma vol(C)^2/(4W^2)
 *               (gamma 0: one community per connected component, 1:
 *               modularity, 2W and above: singletons).  The gain stays an
 *               exact integer, 2W res_den (omega(u,D) - omega(u,C\u)) -
 *               res_num vol(u) (vol(D) - vol(C\u)).  res_num >= 0,
 *               res_den >= 1, reduced by their gcd, and max(res_num,
 *               res_den) (2W)^2 < 2^126, else CD_EINVAL; (0, 0) means 1 / 1.
 *               The reported modularity is always the standard one (gamma 1).
 *               PLP ignores it.
 *   schedule    0 (default): the deterministic colour-class schedule, results
 *               identical to the sequential oracle.  R in 1..4096: the
 *               paper's racy schedule (Sections III-A, III-B) for the PLM
 *               move phases, cut into R rounds: no colouring; a seeded hash
 *               splits the vertices into R rounds, and adjacent vertices may
 *               share one.  In the first four sweeps of a phase every vertex
 *               of a round decides in parallel on the labels and community
 *               volumes as they are at that moment and applies its move at
 *               once.  Later sweeps decide on the round's starting state and
 *               re-check the wanted moves one by one in vertex order; a move
 *               waits for the next sweep when an earlier move of the round
 *               left or entered its current or target community, so every
 *               applied move raises the objective and the phase terminates.
 *               Results depend on the timing of the threads in the first
 *               sweeps and may differ between runs; they are valid partitions
 *               with their exact modularity.  The level loop also stops when
 *               coarsening no longer merges vertices.  PLP and EPP's base runs
 *               keep the colour classes.  128 rounds are the binding's default.
 *   int_path    0 (default): the move gains are computed in 64 bits when
 *               max(res_num, res_den) (2W)^2 < 2^63 and 2W < 2^31, else in 128
 *               bits; 128 forces the 128-bit path (same results); 64 demands
 *               the 64-bit path and fails with CD_EINVAL where it would not be
 *               exact.
 *   scratch_budget  0 (default), or the low-memory mode (the GPU analogue
 *               of the paper's memory-lean PLM*, Section III-B): coarsening,
 *               whose sort scratch otherwise takes about 52 bytes per
 *               inter-community adjacency entry of a level (the largest
 *               working buffer of a run), processes ranges of coarse rows so
 *               that one pass uses at most this many bytes (a single coarse
 *               row above the budget forms a pass of its own).  A level's
 *               schedule (colour classes and hub tables) is also freed once
 *               its move phase is done and rebuilt for PLMR's refinement on
 *               the way up.  Slower, same results.
 * cd_tune picks team_quantum, team_min and bin_max by measurement. */
typedef struct {
    uint64_t seed;
    int32_t max_sweeps;
    int32_t max_levels;
    int32_t max_iters;
    int32_t profile;
    int64_t team_quantum;
    int32_t team_min;
    int32_t reserved;   /* 0 */
    int32_t bin_max[5];
    int64_t res_num;    /* resolution gamma = res_num / res_den of PLM / PLMR */
    int64_t res_den;    /*   and of EPP's final phase (1 / 1: modularity) */
    int32_t schedule;   /* 0: colour classes (deterministic); R >= 1: racy, R rounds */
    int32_t int_path;   /* gain width of PLM: 0 automatic, 64 or 128 */
    int64_t scratch_budget;   /* low-memory mode: bytes of coarsening scratch; 0: none */
} cd_opts;

/* Run statistics (all optional: pass NULL to skip). */
typedef struct {
    int32_t levels;          /* graphs in the hierarchy that ran a move phase */
    int32_t colors0;         /* colour classes of the input level */
    int32_t converged;       /* 1 unless some phase hit its cap */
    int32_t ncomm;           /* communities in the output */
    int64_t sweeps;          /* move sweeps (PLM/PLMR) over all levels */
    int64_t moves;           /* applied moves (PLM) or label updates (PLP) */
    int64_t iters;           /* PLP iterations (EPP: summed over bases) */
    int64_t entries;         /* adjacency entries scanned by decide kernels */
    int64_t candidates;      /* distinct neighbour communities evaluated */
    int64_t decisions;       /* vertex decisions taken */
    double ms_color, ms_move, ms_coarsen, ms_total;
    /* local-move kernels, filled when opts.profile = 1 */
    int64_t k_launches;      /* move-phase / PLP kernel launches timed */
    double k_ms;             /* their summed device time */
    double k_bytes;          /* their algorithmic bytes (from the schedule counters) */
    double stage_items_ms;   /* PLM move kernel: whole class steps (profile mode) */
    double stage_sort_ms;    /*   re-check: sorting the wanted moves by id */
    double stage_recheck_ms; /*   re-check of late sweeps, sort included */
} cd_stats;

void cd_opts_default(cd_opts *o);
const char *cd_status_str(cd_status s);
/* Message of the last failure on the calling thread ("" if none). */
const char *cd_last_error(void);

/* Creates a graph handle: validates the CSR (conventions above), copies it to
 * device memory owned by the handle, stores self-loops apart and computes
 * vol(u) = sum of weights to other vertices + 2 * loop weight and the total
 * weight omega(E) (Section III-B).  `stream` is a cudaStream_t (NULL: the
 * legacy default stream) used by every later call on this handle.
 * mem_flags CD_BORROW: row_ptr, col and w are device arrays that the handle
 * reads in place instead of copying; the caller keeps them alive and
 * unchanged until cd_graph_destroy.  When the graph has self-loops the
 * handle still keeps a copy of the adjacency without them (the kernels read
 * loop-free rows); the input arrays are never duplicated as they are.
 * Errors: CD_EINVAL (bad sizes, unsorted or duplicate columns, column out of
 * range, non-positive weight, asymmetric entry or weight) with nothing
 * allocated; CD_ENOMEM; CD_ECUDA. */
cd_status cd_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const int32_t *w, int mem_flags, void *stream, cd_graph **out);
cd_status cd_graph_destroy(cd_graph *g);
/* n, undirected loop-free edge count m, total weight omega(E). */
cd_status cd_graph_info(const cd_graph *g, int64_t *n, int64_t *m, int64_t *total_weight);

/* Modularity of `labels` (Eq. 1): mod = sum_C omega(C)/omega(E) -
 * vol(C)^2/(4 omega(E)^2), evaluated exactly as the integer fraction
 * N/D with N = 2 omega(E) sum_C 2 omega(C) - sum_C vol(C)^2, D = 4 omega(E)^2,
 * then one IEEE double division.  Labels must lie in [0, n).  0 when the
 * graph has no edges.  Errors: CD_EINVAL (label out of range). */
cd_status cd_modularity(cd_graph *g, const int32_t *labels, int labels_mem, double *mod);

/* PLP, Algorithm 1: from singletons, each vertex with an active flag and a
 * non-loop neighbour adopts the dominant neighbour label (largest summed edge
 * weight) when it is strictly heavier than its current label; ties between
 * dominant labels follow a seeded pseudo-random order.  Iterates while more
 * than `theta` vertices changed (theta < 0: n * 1e-5, Section III-A).
 * Vertices are visited in colour classes; an update re-activates the
 * neighbours, a non-update deactivates the vertex. */
cd_status cd_plp(cd_graph *g, const cd_opts *o, double theta, int32_t *labels,
                 int labels_mem, double *mod, cd_stats *st);

/* PLM (Algorithm 3) or, with refine = 1, PLMR (Algorithm 4).  Move phase
 * (Algorithm 2): in colour classes, every vertex u picks the neighbour
 * community D maximising the exact gain
 *   g = 2W (omega(u,D) - omega(u,C\u)) - vol(u) (vol(D) - vol(C\u))
 * (Delta mod of Section III-B times 2W^2; ties to the smallest id) and moves
 * if g > 0; sweeps repeat until no vertex wants to move.  If anything moved,
 * the graph is coarsened by communities and solved recursively, and the
 * coarse solution is prolonged (PLMR: followed by another move phase). */
cd_status cd_plm(cd_graph *g, int refine, const cd_opts *o, int32_t *labels,
                 int labels_mem, double *mod, cd_stats *st);

/* EPP(b, PLP, Final), Algorithm 5: b PLP runs (run i seeded seed+i), their
 * core communities (Eq. 2: same core iff same community in every run),
 * coarsening by the cores, Final = PLM (final_refine 0) or PLMR (1) on the
 * core graph, prolongation.  b >= 1. */
cd_status cd_epp(cd_graph *g, int ensemble_size, int final_refine, const cd_opts *o,
                 int32_t *labels, int labels_mem, double *mod, cd_stats *st);

/* EPP(b, Base, Final) of Section III-D, which leaves the base and final
 * algorithms open, with iterated ensembles (the hierarchy of core graphs of
 * the scheme EPP adapts, Section II).  base: CD_BASE_PLP, CD_BASE_PLM or
 * CD_BASE_PLMR; Final = PLM (final_refine 0) or PLMR (1).  Round r = 0, 1,
 * ..., rounds - 1 runs the b base algorithms on the current graph (run i
 * seeded seed + r b + i), forms their core communities (Eq. 2) and coarsens
 * by them.  Round 0 is Algorithm 5; a later round is taken only if its core
 * merges vertices and has strictly higher modularity than the previous
 * round's core, else the rounds stop.  The final algorithm runs on the last
 * core graph (seed), and its labels are prolonged to the input graph.
 * cd_stats.levels is the number of core graphs taken.  base = CD_BASE_PLP
 * with rounds = 1 is cd_epp.  b >= 1, 1 <= rounds <= 64, else CD_EINVAL. */
enum { CD_BASE_PLP = 0, CD_BASE_PLM = 1, CD_BASE_PLMR = 2 };
cd_status cd_epp_general(cd_graph *g, int ensemble_size, int base, int final_refine, int rounds,
                         const cd_opts *o, int32_t *labels, int labels_mem, double *mod, cd_stats *st);

/* Batched and served runs.  The paper runs one graph at a time; its only
 * multi-instance notion is the nested parallelism of EPP's base runs
 * (Section III-C).  Here many runs share the GPU: each run advances through
 * the same stages as the single-graph call (on host worker threads), and the
 * persistent phases (PLM move phases, PLP runs) pending at the same moment
 * share one cooperative launch, in which teams of blocks pull graphs from a
 * device queue.  Batching changes nothing observable: every run's labels,
 * modularity and statistics equal those of the single-graph call with the
 * same task and options. */

enum { CD_ALGO_PLP = 0, CD_ALGO_PLM = 1, CD_ALGO_EPP = 2 };

/* What to run on a graph. */
typedef struct {
    int32_t algo;       /* CD_ALGO_PLP, CD_ALGO_PLM or CD_ALGO_EPP */
    int32_t refine;     /* PLM: 1 = PLMR; EPP: 1 = PLMR as the final algorithm */
    int32_t ensemble;   /* EPP: number of PLP base runs b >= 1 */
    int32_t reserved;   /* 0 */
    double theta;       /* PLP: iteration threshold (< 0: n * 1e-5); EPP bases always use n * 1e-5 */
} cd_task;

/* Runs `task` on `count` graphs together.
 *   gs          count graph handles (a handle may repeat); their streams are
 *               synchronised on entry
 *   labels      count pointers; labels[i] holds n_i entries in labels_mem memory
 *   mods        NULL or double[count]
 *   st          NULL or cd_stats[count]
 *   stream      cudaStream_t of the batched launches (NULL: legacy default)
 * Synchronous.  Up to 16 host threads advance the runs between launches.
 * Errors: after every run has stopped, the status of the first failing run
 * in order (CD_EINVAL for bad arguments before anything runs); CD_ENOTCONV
 * when some run hit its cap (results still valid). */
cd_status cd_run_batch(cd_graph *const *gs, int count, const cd_task *task, const cd_opts *o,
                       int32_t *const *labels, int labels_mem, double *mods, cd_stats *st, void *stream);

/* Launch-shape autotuner: runs `task` on the count graphs (together, as
 * cd_run_batch does, when count > 1) under candidate values of team_quantum,
 * team_min (only when launches are shared: count > 1 or EPP) and bin_max,
 * one option at a time, keeping a candidate when its complete run is at
 * least 1% faster than the current choice, until max_trials runs have been
 * made.  *best receives `base` (NULL: defaults) with the chosen shape and
 * *best_ms (may be NULL) the wall time of its run.  These options never
 * change results, so tuning is safe on the caller's own workload.
 * Synchronous.  Errors: CD_EINVAL, then those of the runs. */
cd_status cd_tune(cd_graph *const *gs, int count, const cd_task *task, const cd_opts *base, int max_trials,
                  cd_opts *best, double *best_ms, void *stream);

/* cd_run_batch of PLM (refine 0) or PLMR (refine 1) on the stream of gs[0]. */
cd_status cd_plm_batch(cd_graph *const *gs, int count, int refine, const cd_opts *o,
                       int32_t *const *labels, int labels_mem, double *mods, cd_stats *st);

/* Server: continuous batching of submitted runs in two lanes, small runs
 * (adjacency entries plus vertices up to 2^21) and large runs.  Each lane is
 * a host thread with its own stream.  Small runs' launches use a quarter of
 * the device's resident blocks, large runs' launches the rest while small
 * runs are active and the whole device otherwise, so the lanes' launches run
 * side by side and a small run does not wait for a large run's phases.  A lane admits
 * its queued runs in submission order while at most max_slots runs (both
 * lanes together) are admitted and their estimated device memory stays within
 * device_mem_budget bytes (0: 80% of the device memory free at creation).  An
 * admitted run joins its lane's next batched launch, so runs submitted while
 * others are on the GPU overlap with them; a finished run frees its slot and
 * memory at once.  Graphs, labels and volumes of every level stay on the
 * device for the whole run.
 *   max_queue   submitted runs not yet admitted, at most (CD_EBUSY beyond)
 *   stream      cudaStream_t of the large lane's launches (NULL: the server
 *               creates its own; the small lane always has its own) */
cd_status cd_server_create(size_t device_mem_budget, int max_slots, int max_queue, void *stream, cd_server **out);
/* Queues `task` on g; g must stay alive until the run's result is taken.
 * ticket receives the run's id.  Errors: CD_EBUSY (queue full), CD_EINVAL
 * (bad task, or a run that could never fit the budget). */
cd_status cd_server_submit(cd_server *s, cd_graph *g, const cd_task *task, const cd_opts *o, uint64_t *ticket);
/* Takes a finished run's result: labels (n entries, labels_mem memory; NULL
 * to skip), modularity, latency from submission to completion in ms, stats
 * (each may be NULL); the ticket is then released.  Waits at most timeout_ms
 * (0: do not wait; < 0: no limit).  Returns CD_EBUSY while the run is queued
 * or running when the wait ends, CD_EINVAL for an unknown ticket, otherwise
 * the run's own status. */
cd_status cd_server_poll(cd_server *s, uint64_t ticket, double timeout_ms, int32_t *labels, int labels_mem,
                         double *mod, double *latency_ms, cd_stats *st);
/* Counters: runs queued, running and finished but not yet taken. */
cd_status cd_server_info(cd_server *s, int64_t *queued, int64_t *running, int64_t *finished);
/* Stops admitting, lets the runs on the GPU finish their current launch,
 * drops every unfinished run and frees everything. */
cd_status cd_server_destroy(cd_server *s);

/* Building blocks exposed for verification. */

/* Colour classes used as the schedule: first-fit Jones-Plassmann colouring
 * with priorities (fmix32(v ^ fmix32(seed_lo ^ seed_hi)), v).  colors[n]. */
cd_status cd_color(cd_graph *g, uint64_t seed, int32_t *colors, int colors_mem,
                   int32_t *ncolors);

/* Coarsening (Section III-B, coarsen): one coarse vertex per distinct label
 * (numbered by ascending label), inter-community weights summed, the
 * intra-community weight kept as the coarse self-loop.  Returns a new graph
 * handle (int64 weights) on the same stream.  Labels in [0, n). */
cd_status cd_coarsen(cd_graph *g, const int32_t *labels, int labels_mem, cd_graph **coarse);

/* Copies a handle's graph out in input-CSR form: row_ptr[n+1], col[nnz],
 * w[nnz] as int64 (self-loop once in its row).  nnz_out receives the entry
 * count; pass NULL arrays to query it first.  Host or device buffers. */
cd_status cd_graph_export(const cd_graph *g, int64_t *row_ptr, int32_t *col, int64_t *w,
                          int mem, int64_t *nnz_out);

/* Modularity (as cd_modularity) of `labels` on a CSR that the caller keeps
 * in device memory, computed without allocating any device memory.  The
 * paper has no counterpart: this serves callers that must not allocate when
 * they ask, such as code running inside a device-memory budget another
 * framework owns, latency-critical loops that may not reach the allocator
 * (an allocation can synchronise the device), or hooks run where allocation
 * is not permitted.
 *   n, row_ptr, col, w   the graph in the input conventions above (device
 *                        pointers; w may be NULL for unit weights, col may
 *                        be NULL when the graph has no entries); n must
 *                        not exceed 1,048,576
 *   labels               device int32[n], each in [0, n) (may be NULL when
 *                        n = 0); an edgeless graph has modularity 0
 *   stream               cudaStream_t to run on (NULL: legacy default)
 *   mod                  host double receiving the result
 * Scratch is one fixed device array in the library (8.4 MB, held on every GPU
 * that loads the library until the process exits).  The first call on a device
 * looks up that array's address with the device current, so make it before
 * any stream capture.  Calls share the array: each call clears what must
 * start at zero, and calls that overlap on the GPU race, so serialise them.
 * Synchronous.  Errors: CD_EINVAL (n too large, NULL pointer, column or label
 * out of range, non-positive weight, bad row_ptr), CD_ECUDA. */
cd_status cd_modularity_static(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                               const int32_t *labels, void *stream, double *mod);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all devices). */
uint64_t cd_launch_count(void);

/* Device memory of the library's pool on the current device, in bytes: in
 * use now, the high-water mark of use since the last reset (reset_high != 0
 * restarts it after reading), and reserved from the driver (freed memory
 * stays reserved for later runs).  Any pointer may be NULL.  Errors:
 * CD_ECUDA. */
cd_status cd_memory_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, int reset_high);

/* Testing hook: the k-th device allocation from now fails with CD_ENOMEM
 * (k <= 0 disables).  Used to check that failures leak nothing. */
void cd_debug_fail_alloc(int k);

/* Testing hook: the batch engine's launch planner (cd_run_batch, Section
 * III-C's nested parallelism as one launch) on bare phase sizes, on the host
 * only (no device work, no GPU needed).  work[i] (count >= 1 entries) is the
 * adjacency entries plus vertices of run i; team_quantum and team_min are the
 * cd_opts fields of that name; grid_max is the number of resident blocks.
 * Writes the grid used (<= grid_max), the number of tiers (<= 16), six int32
 * per tier into tiers[16 * 6] (first block, blocks, team size, index of the
 * first team, first run in `order`, number of runs), and in order[count] the
 * runs in tier order.  Errors: CD_EINVAL. */
cd_status cd_debug_plan_launch(const int64_t *work, int count, int64_t team_quantum, int32_t team_min, int grid_max,
                               int32_t *grid, int32_t *ntiers, int32_t *tiers, int32_t *order);

/* Diagnostic: the class trace of the move phases (Algorithm 2 under the
 * colour-class schedule) run with opts.profile = 2 since the last call.  One
 * row of nineteen int64 per class step, in completion order: phase number,
 * sweep, colour class, its vertices, its adjacency entries, its hub
 * aggregation chunks, its hub decide slices, its hubs above 4096 neighbours,
 * the wall time in ns on the team's first block from the previous class's
 * barrier to this class's barrier, the latest times (ns after that start, 0
 * when absent) at which a block finished its work items, its hub decide
 * slices, and the class finisher its work, and at which a block began its
 * first item; the longest single lane-group item, block item and hub-chunk
 * item, the longest wait of a decide slice for its hub's table and the
 * longest decide slice after it (ns); the class's applied moves (early
 * sweeps) or re-check candidates (late sweeps).  With out == NULL only
 * *count (rows) is set; then out[19 * count] receives the rows (cap = rows
 * the buffer holds) and the trace is cleared.  Errors: CD_EINVAL. */
cd_status cd_debug_class_trace(int64_t *out, int64_t cap, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif /* CD_H */
