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

enum { CD_MEM_HOST = 0, CD_MEM_DEVICE = 1 };

/* Options.  cd_opts_default() fills: seed 1, max_sweeps 256, max_levels 64,
 * max_iters 1000, profile 0.
 *   seed        colouring priorities (Jones-Plassmann), PLP tie order and the
 *               move-damping coin all derive from it; EPP base i uses seed+i.
 *   max_sweeps  cap on sweeps of one move phase (Algorithm 2 "repeat").
 *   max_levels  cap on the coarsening hierarchy depth (Algorithm 3).
 *   max_iters   cap on PLP iterations (Algorithm 1 "while").
 *   profile     1: time every local-move kernel launch with CUDA events and
 *               report it in cd_stats (adds host synchronisation). */
typedef struct {
    uint64_t seed;
    int32_t max_sweeps;
    int32_t max_levels;
    int32_t max_iters;
    int32_t profile;
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
    double stage_items_ms;   /* PLM move kernel: decide items of each class */
    double stage_hub_ms;     /*   hub decisions */
    double stage_recheck_ms; /*   sequential re-check of late sweeps */
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
 *                        pointers; w may be NULL for unit weights); n must
 *                        not exceed 1,048,576
 *   labels               device int32[n], each in [0, n)
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

/* Testing hook: the k-th device allocation from now fails with CD_ENOMEM
 * (k <= 0 disables).  Used to check that failures leak nothing. */
void cd_debug_fail_alloc(int k);

#ifdef __cplusplus
}
#endif
#endif /* CD_H */
