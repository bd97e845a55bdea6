/*
 * Reference oracle for PLP / PLM / PLMR / EPP community detection
 * (Staudt & Meyerhenke, "Engineering Parallel Algorithms for Community
 * Detection in Massive Networks").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential CPU
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may build, load or call it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * Arithmetic is exact: weights, volumes and sums in int64, every product of
 * the modularity gain and of the modularity numerator in __int128, and one
 * final IEEE double division for modularity.
 *
 * Readings of the paper that the code fixes (the paper is silent or the
 * parallel schedule is nondeterministic there):
 *   - vol(u) sums the weights to neighbours other than u plus twice the
 *     self-loop (Section III-B, volume definition; read so that sum vol = 2W).
 *   - Schedule: colour classes of a hash-priority Jones-Plassmann colouring
 *     (computed in one pass as greedy colouring in descending priority
 *     order, which it equals), processed in ascending colour; inside a class every vertex decides on
 *     the labels and community volumes as they stood when the class began,
 *     then all decisions of the class are applied.  The colouring ignores
 *     edges between two hubs (vertices with more than HUB_RELAX neighbours),
 *     so adjacent hubs may share a class and then decide on each other's
 *     labels from the start of the class: one instance of the stale data the
 *     paper's parallel threads work with (Section III-B).
 *   - Ties in the argmax of the move rule go to the smallest community id;
 *     a move needs a strictly positive gain (Algorithm 2).  A move phase
 *     ends when no vertex wants to move; from its 5th sweep on, the wanted
 *     moves of a class are re-checked one by one in vertex order against
 *     the volumes already updated, and a hub whose current or target
 *     community a hub accepted earlier in the class left or entered is
 *     passed over (see move_phase).
 *   - PLP adopts the dominant label only if its weight strictly exceeds the
 *     weight of the current label; ties between dominant labels follow a
 *     per-iteration pseudo-random order of the labels (fmix32 of the label
 *     xor a salt drawn from the seed and the iteration number).  Hubs are
 *     evaluated in every iteration (active or not; the active set never
 *     changes a result).
 *   - Every recursive PLM/PLMR call returns a compacted labelling (dense
 *     ranks in ascending order of raw label); prolongation works in that
 *     space.
 *   - EPP base run i colours with seed+i; the combination is the exact
 *     core-community partition of Eq. (2) (pairwise key compaction), not a
 *     hash.
 *   - The resolution gamma of Section III-B scales the volume term of the
 *     move gain; it is a rational p/q (default 1/1, modularity) so that the
 *     gain stays an exact integer, and the reported quality stays the
 *     standard modularity.
 *   - Caps: 256 sweeps per move phase, 64 levels, 1000 PLP iterations.
 *   - Modularity of an edgeless graph is 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* Built twice: plain (sequential) and with -fopenmp.  The OpenMP build runs
 * the decisions of one colour class in parallel, which the schedule makes
 * independent of each other (every vertex of a class reads only labels and
 * volumes fixed before the class; Section III-B's parallel loop over the
 * vertices).  Everything else runs in the same order in both builds, so the
 * two give identical results. */
#ifdef _OPENMP
#include <omp.h>
#define OR_THREADS() omp_get_max_threads()
#define OR_TID() omp_get_thread_num()
#else
#define OR_THREADS() 1
#define OR_TID() 0
#endif
/* classes with fewer adjacency entries than this are decided by one thread */
#define OR_PAR_MIN 4096

/* adjacency entries of the vertices v[a..b) (the work of deciding them) */
#define CLASS_WORK(g, v, a, b, out) do {                                       \
        int64_t w_ = 0;                                                         \
        for (int64_t i_ = (a); i_ < (b); i_++)                                  \
            w_ += (g)->rp[(v)[i_] + 1] - (g)->rp[(v)[i_]];                      \
        (out) = w_;                                                             \
    } while (0)

/* Hubs for the colouring: more than HUB_RELAX neighbours (self-loop not
 * counted).  Edges between two hubs do not constrain the colouring. */
#define HUB_RELAX 4096

/* ---------------------------------------------------------------------- */
/* Graph: adjacency without self-loops, self-loop weights kept apart.       */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    int64_t *rp;    /* [n+1] row offsets into adj/wt */
    int32_t *adj;   /* neighbours v != u */
    int64_t *wt;    /* weight of {u, v} */
    int64_t *loop;  /* [n] self-loop weight omega(u, u) */
    int64_t *vol;   /* [n] vol(u) */
    int64_t W;      /* omega(E): every edge once, self-loops once */
    int64_t res_num, res_den;   /* resolution gamma = res_num / res_den of the
                                 * move gain (Sec. III-B); 1/1: modularity */
} OG;

static void og_free(OG *g)
{
    free(g->rp); free(g->adj); free(g->wt); free(g->loop); free(g->vol);
    memset(g, 0, sizeof(*g));
}

/* vol(u) and omega(E) from their definitions (Section III-B). */
static void og_volumes(OG *g)
{
    int64_t twice = 0;
    for (int64_t u = 0; u < g->n; u++) {
        int64_t s = 2 * g->loop[u];
        for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) s += g->wt[e];
        g->vol[u] = s;
        twice += s;
    }
    g->W = twice / 2;
}

/* Input CSR (self-loop stored once in its row) -> OG.  w == NULL: unit. */
static int og_from_input(OG *g, int64_t n, const int64_t *row_ptr,
                         const int32_t *col, const int64_t *w)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->res_num = g->res_den = 1;
    g->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->loop = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->vol = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t nnz = row_ptr[n];
    g->adj = (int32_t *)malloc(((size_t)nnz + 1) * sizeof(int32_t));
    g->wt = (int64_t *)malloc(((size_t)nnz + 1) * sizeof(int64_t));
    if (!g->rp || !g->loop || !g->vol || !g->adj || !g->wt) { og_free(g); return -1; }
    int64_t k = 0;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int64_t wt = w ? w[e] : 1;
            if (col[e] == u) g->loop[u] += wt;
            else { g->adj[k] = col[e]; g->wt[k] = wt; k++; }
        }
        g->rp[u + 1] = k;
    }
    og_volumes(g);
    return 0;
}

/* Resolution gamma = p/q of the move gain (Section III-B).  The fraction is
 * reduced by gcd(p, q), which scales every gain by one positive factor and
 * so changes no decision.  Both products of the gain are bounded by
 * max(p, q) (2W)^2 (|omega(u,D) - omega(u,C\u)|, vol(u) and |vol(D) -
 * vol(C\u)| are at most 2W), so p/q is accepted only when that bound stays
 * below 2^126 and the gain fits a signed 128-bit integer.  Returns -2 for
 * p < 0, q < 1 or a fraction outside that range. */
static int og_set_resolution(OG *g, int64_t p, int64_t q)
{
    if (p < 0 || q < 1) return -2;
    int64_t a = p, b = q;
    while (b) { int64_t t = a % b; a = b; b = t; }
    if (a > 1) { p /= a; q /= a; }
    const i128 w2 = (i128)(2 * g->W) * (2 * g->W);
    const i128 lim = ((i128)1) << 126;
    const int64_t big = p > q ? p : q;
    if (w2 > 0 && (i128)big > (lim - 1) / w2) return -2;
    g->res_num = p;
    g->res_den = q;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Modularity, Eq. (1):                                                     */
/*   mod = sum_C omega(C)/W - vol(C)^2/(4 W^2)                              */
/* written over the common denominator 4W^2:                                */
/*   N = 2W * sum_C 2 omega(C) - sum_C vol(C)^2,  D = 4 W^2.                */
/* ---------------------------------------------------------------------- */
static void og_mod_num(const OG *g, const int32_t *z, i128 *N, i128 *D)
{
    int64_t in2 = 0;  /* sum_C 2 omega(C) */
    int64_t *volc = (int64_t *)calloc((size_t)g->n + 1, sizeof(int64_t));
    for (int64_t u = 0; u < g->n; u++) {
        in2 += 2 * g->loop[u];
        for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++)
            if (z[g->adj[e]] == z[u]) in2 += g->wt[e];
        volc[z[u]] += g->vol[u];
    }
    i128 sq = 0;
    for (int64_t c = 0; c < g->n; c++) sq += (i128)volc[c] * volc[c];
    free(volc);
    *N = (i128)(2 * g->W) * in2 - sq;
    *D = (i128)4 * g->W * g->W;
}

static double og_modularity(const OG *g, const int32_t *z)
{
    if (g->W == 0) return 0.0;
    i128 N, D;
    og_mod_num(g, z, &N, &D);
    return (double)N / (double)D;
}

/* ---------------------------------------------------------------------- */
/* Compaction: dense rank of each label in ascending order of raw label.    */
/* Labels are in [0, n).                                                     */
/* ---------------------------------------------------------------------- */
static int64_t dense_rank(int64_t n, const int32_t *z, int32_t *rank_of_label)
{
    char *used = (char *)calloc((size_t)n + 1, 1);
    for (int64_t u = 0; u < n; u++) used[z[u]] = 1;
    int64_t k = 0;
    for (int64_t l = 0; l < n; l++) rank_of_label[l] = used[l] ? (int32_t)k++ : -1;
    free(used);
    return k;
}

static int64_t compact(int64_t n, int32_t *z)
{
    int32_t *rk = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t k = dense_rank(n, z, rk);
    for (int64_t u = 0; u < n; u++) z[u] = rk[z[u]];
    free(rk);
    return k;
}

/* ---------------------------------------------------------------------- */
/* Colouring: first-fit Jones-Plassmann with hash priorities on the graph    */
/* without its hub-hub edges.                                               */
/* Priority of v: (fmix32(v ^ fmix32(seed_lo ^ seed_hi)), v), compared      */
/* lexicographically, larger wins.  fmix32 is the MurmurHash3 32-bit        */
/* finaliser (Appleby).                                                     */
/* ---------------------------------------------------------------------- */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16; h *= 0x85ebca6bu;
    h ^= h >> 13; h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static int prio_greater(const uint32_t *h, int32_t a, int32_t b)
{
    return h[a] > h[b] || (h[a] == h[b] && a > b);
}

static int is_hub(const OG *g, int32_t v)
{
    return g->rp[v + 1] - g->rp[v] > HUB_RELAX;
}

static int32_t color_jp(const OG *g, uint64_t seed, int32_t *color)
{
    int64_t n = g->n;
    uint32_t s = fmix32((uint32_t)seed ^ (uint32_t)(seed >> 32));
    uint32_t *h = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    int32_t *pick = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    char *taken = NULL;
    int64_t taken_cap = 0;
    for (int64_t v = 0; v < n; v++) { h[v] = fmix32((uint32_t)v ^ s); color[v] = -1; }
    int64_t left = n;
    int32_t ncol = 0;
    while (left > 0) {
        /* 1. every uncoloured vertex that beats all uncoloured neighbours */
        int64_t np = 0;
        for (int64_t v = 0; v < n; v++) {
            if (color[v] >= 0) continue;
            int best = 1;
            const int vh = is_hub(g, (int32_t)v);
            for (int64_t e = g->rp[v]; e < g->rp[v + 1] && best; e++) {
                int32_t x = g->adj[e];
                if (vh && is_hub(g, x)) continue;
                if (color[x] < 0 && prio_greater(h, x, (int32_t)v)) best = 0;
            }
            if (best) pick[np++] = (int32_t)v;
        }
        /* 2. they are pairwise non-adjacent, hub pairs aside: give each the
         *    smallest colour not used by its neighbours coloured in earlier
         *    rounds (hub neighbours of a hub do not count) */
        for (int64_t i = 0; i < np; i++) {
            int32_t v = pick[i];
            int64_t deg = g->rp[v + 1] - g->rp[v];
            if (deg + 1 > taken_cap) {
                taken_cap = deg + 1;
                taken = (char *)realloc(taken, (size_t)taken_cap);
            }
            memset(taken, 0, (size_t)deg + 1);
            const int vh = is_hub(g, v);
            for (int64_t e = g->rp[v]; e < g->rp[v + 1]; e++) {
                if (vh && is_hub(g, g->adj[e])) continue;
                int32_t c = color[g->adj[e]];
                if (c >= 0 && c <= deg) taken[c] = 1;
            }
            int32_t c = 0;
            while (taken[c]) c++;
            color[v] = c;
            if (c + 1 > ncol) ncol = c + 1;
        }
        left -= np;
    }
    free(h); free(pick); free(taken);
    return ncol;
}

/* The same colouring in one pass.  A Jones-Plassmann round colours a vertex
 * exactly when every neighbour of higher priority is coloured and never
 * before, and first fit looks only at coloured neighbours, so the rounds give
 * the colouring of the sequential greedy method run in descending priority
 * order (each vertex takes the smallest colour its already coloured
 * neighbours leave free; hub-hub edges skipped as above).  This form costs
 * one sort plus one read of every adjacency entry, against one rescan of
 * every uncoloured vertex per round for color_jp. */
static int cmp_u64_desc(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x < y) - (x > y);
}

static int32_t color_greedy(const OG *g, uint64_t seed, int32_t *color)
{
    int64_t n = g->n;
    uint32_t s = fmix32((uint32_t)seed ^ (uint32_t)(seed >> 32));
    uint64_t *key = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    for (int64_t v = 0; v < n; v++) {
        key[v] = ((uint64_t)fmix32((uint32_t)v ^ s) << 32) | (uint32_t)v;
        color[v] = -1;
    }
    qsort(key, (size_t)n, sizeof(uint64_t), cmp_u64_desc);
    char *taken = NULL;
    int64_t taken_cap = 0;
    int32_t ncol = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t v = (int32_t)(uint32_t)key[i];
        int64_t deg = g->rp[v + 1] - g->rp[v];
        if (deg + 1 > taken_cap) {
            taken_cap = deg + 1;
            taken = (char *)realloc(taken, (size_t)taken_cap);
        }
        memset(taken, 0, (size_t)deg + 1);
        const int vh = is_hub(g, v);
        for (int64_t e = g->rp[v]; e < g->rp[v + 1]; e++) {
            if (vh && is_hub(g, g->adj[e])) continue;
            int32_t c = color[g->adj[e]];
            if (c >= 0 && c <= deg) taken[c] = 1;
        }
        int32_t c = 0;
        while (taken[c]) c++;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(key); free(taken);
    return ncol;
}

/* Vertices grouped by colour, ascending id inside a class (or descending
 * when rev != 0: the result must not depend on it). */
typedef struct { int32_t ncol; int64_t *off; int32_t *v; } Classes;

static void classes_build(const OG *g, uint64_t seed, int rev, Classes *cl)
{
    int64_t n = g->n;
    int32_t *color = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    cl->ncol = n ? color_greedy(g, seed, color) : 0;
    cl->off = (int64_t *)calloc((size_t)cl->ncol + 2, sizeof(int64_t));
    cl->v = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    for (int64_t u = 0; u < n; u++) cl->off[color[u] + 1]++;
    for (int32_t c = 0; c < cl->ncol; c++) cl->off[c + 1] += cl->off[c];
    int64_t *pos = (int64_t *)malloc(((size_t)cl->ncol + 1) * sizeof(int64_t));
    memcpy(pos, cl->off, (size_t)cl->ncol * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t u = rev ? n - 1 - i : i;
        cl->v[pos[color[u]]++] = (int32_t)u;
    }
    free(pos); free(color);
}

static void classes_free(Classes *cl) { free(cl->off); free(cl->v); }

/* ---------------------------------------------------------------------- */
/* Statistics                                                                */
/* ---------------------------------------------------------------------- */
enum {
    ST_LEVELS = 0, ST_SWEEPS, ST_MOVES, ST_COLORS0, ST_CONVERGED, ST_ENTRIES,
    ST_CANDIDATES, ST_DECISIONS, ST_ITERS, ST_NCOMM, ST_SWEEPS0, ST_ENTRIES0,
    ST_CANDIDATES0, ST_N
};

/* per-thread counter rows of the OpenMP build, padded to 256 bytes so that
 * two threads never write the same cache line */
#define ST_PAD 32

/* ---------------------------------------------------------------------- */
/* Local moving, Algorithm 2, under the colour-class schedule.               */
/* ---------------------------------------------------------------------- */
typedef struct { int64_t *acc; int32_t *touched; } Scratch;

/* omega(u, c) for every community c adjacent to u (u itself excluded);
 * returns the number of distinct communities, listed in s->touched. */
static int64_t gather_weights(const OG *g, const int32_t *z, int64_t u, Scratch *s)
{
    int64_t nt = 0;
    for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
        int32_t c = z[g->adj[e]];
        if (s->acc[c] == 0) s->touched[nt++] = c;
        s->acc[c] += g->wt[e];
    }
    return nt;
}

static void clear_weights(Scratch *s, int64_t nt)
{
    for (int64_t i = 0; i < nt; i++) s->acc[s->touched[i]] = 0;
}

/* Gain of moving u from C = z[u] to D != C, multiplied by 2W^2 > 0
 * (Section III-B, Delta mod):
 *   g = 2W (omega(u,D) - omega(u,C\u)) - vol(u) (vol(D) - vol(C\u)).
 * With a resolution gamma = p/q (Section III-B: gamma scales the volume
 * term; 0 yields one community per connected component, 1 is modularity,
 * 2W yields singletons) the gain is multiplied by 2W^2 q instead:
 *   g = 2W q (omega(u,D) - omega(u,C\u)) - p vol(u) (vol(D) - vol(C\u)). */
static i128 gain(const OG *g, int64_t w_uD, int64_t w_uC, int64_t vol_u,
                 int64_t vol_D, int64_t vol_C)
{
    return (i128)g->res_den * (2 * g->W) * (w_uD - w_uC)
         - (i128)g->res_num * vol_u * (vol_D - (vol_C - vol_u));
}

/* Best target community for u, or z[u] if no candidate has positive gain. */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int32_t decide_move(const OG *g, const int32_t *z, const int64_t *volc,
                           int64_t u, Scratch *s, int64_t st[ST_N], int level0,
                           int64_t *out_wD, int64_t *out_wC)
{
    int64_t nt = gather_weights(g, z, u, s);
    int32_t C = z[u];
    int64_t w_uC = s->acc[C];
    int32_t best = C;
    i128 bestg = 0;
    int have = 0;
    for (int64_t i = 0; i < nt; i++) {
        int32_t D = s->touched[i];
        if (D == C) continue;
        i128 gD = gain(g, s->acc[D], w_uC, g->vol[u], volc[D], volc[C]);
        if (!have || gD > bestg || (gD == bestg && D < best)) { best = D; bestg = gD; have = 1; }
    }
    st[ST_ENTRIES] += g->rp[u + 1] - g->rp[u];
    st[ST_CANDIDATES] += nt;
    st[ST_DECISIONS] += (g->rp[u + 1] > g->rp[u]);   /* vertices with neighbours */
    if (level0) {
        st[ST_ENTRIES0] += g->rp[u + 1] - g->rp[u];
        st[ST_CANDIDATES0] += nt;
    }
    *out_wD = have ? s->acc[best] : 0;    /* omega(u, D) of the chosen target */
    *out_wC = w_uC;                       /* omega(u, C \ u) */
    clear_weights(s, nt);
    return (have && bestg > 0) ? best : C;
}

/* Sweeps over the colour classes until no vertex wants to move (zeta is
 * stable, Algorithm 2) or max_sweeps is reached.  Returns the number of
 * moves made.
 *
 * All vertices of a class decide on the volume snapshot taken when the class
 * begins.  In the first RECHECK_FROM sweeps every wanted move of the class is
 * applied.  Simultaneous moves into (or out of) one community can overshoot,
 * since each assumed the others stay put, and on some graphs that churn does
 * not die out.  From sweep RECHECK_FROM on, the wanted moves of a class are
 * applied one at a time in ascending vertex id, each only if its gain,
 * recomputed with the volumes as updated by the moves applied before it, is
 * still positive (its target stays the one it chose).  Vertices of a class
 * are pairwise non-adjacent except hub pairs.  A hub moved in this class
 * changes omega(v, .) of an adjacent hub v only for the two communities it
 * left and entered, so a hub whose own current or target community is one
 * of those is passed over; the omega terms of every accepted move are then
 * exact, only the volume terms interact, each applied move raises
 * modularity by its recomputed gain, and the phase must terminate.
 * The paper lets concurrent threads work on stale data and reports that
 * termination was never a problem in practice (Section III-B). */
#define RECHECK_FROM 4

static int64_t move_phase(const OG *g, int32_t *z, const Classes *cl, uint64_t seed,
                          int32_t max_sweeps, int64_t st[ST_N], int level0)
{
    (void)seed;
    int64_t n = g->n;
    int64_t *volc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *prop = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t *wprop = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t *wcur = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t *byid = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    const int T = OR_THREADS();
    Scratch *ts = (Scratch *)calloc((size_t)T, sizeof(Scratch));
    int64_t (*tst)[ST_PAD] = calloc((size_t)T, sizeof(*tst));  /* per-thread counters */
    for (int t = 0; t < T; t++) {
        ts[t].acc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        ts[t].touched = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    }
    for (int64_t u = 0; u < n; u++) volc[z[u]] += g->vol[u];
    /* stamp[X] = class step in which a hub moved into or out of community X */
    int64_t *stamp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    for (int64_t u = 0; u < n; u++) stamp[u] = -1;
    int64_t step = 0;
    int64_t total = 0;
    int converged = 0;
    for (int32_t sw = 0; sw < max_sweeps; sw++) {
        int64_t wanted = 0, moved = 0;
        for (int32_t k = 0; k < cl->ncol; k++) {
            int64_t a = cl->off[k], b = cl->off[k + 1];
            step++;
            int64_t work;
            CLASS_WORK(g, cl->v, a, b, work);
            (void)work;
            #pragma omp parallel for schedule(dynamic, 16) if (work >= OR_PAR_MIN)
            for (int64_t i = a; i < b; i++) {            /* decide */
                int32_t u = cl->v[i];
                const int t = OR_TID();
                prop[u] = decide_move(g, z, volc, u, &ts[t], tst[t], level0, &wprop[u], &wcur[u]);
            }
            if (sw < RECHECK_FROM) {
                for (int64_t i = a; i < b; i++) {        /* apply all */
                    int32_t u = cl->v[i];
                    if (prop[u] == z[u]) continue;
                    wanted++;
                    volc[z[u]] -= g->vol[u];
                    volc[prop[u]] += g->vol[u];
                    z[u] = prop[u];
                    moved++;
                }
            } else {
                int64_t nc = 0;                          /* wanted moves by id */
                for (int64_t i = a; i < b; i++)
                    if (prop[cl->v[i]] != z[cl->v[i]]) byid[nc++] = cl->v[i];
                qsort(byid, (size_t)nc, sizeof(int32_t), cmp_i32);
                wanted += nc;
                for (int64_t j = 0; j < nc; j++) {
                    int32_t u = byid[j], C = z[u], D = prop[u];
                    /* a hub whose omega(u, C) or omega(u, D) a hub moved
                     * earlier in this class may have changed waits for the
                     * next sweep */
                    const int uh = is_hub(g, u);
                    if (uh && (stamp[C] == step || stamp[D] == step)) continue;
                    if (gain(g, wprop[u], wcur[u], g->vol[u], volc[D], volc[C]) <= 0) continue;
                    volc[C] -= g->vol[u];
                    volc[D] += g->vol[u];
                    z[u] = D;
                    moved++;
                    if (uh) { stamp[C] = step; stamp[D] = step; }
                }
            }
        }
        st[ST_SWEEPS]++;
        if (level0) st[ST_SWEEPS0]++;
        total += moved;
        if (wanted == 0) { converged = 1; break; }
    }
    if (!converged) st[ST_CONVERGED] = 0;
    st[ST_MOVES] += total;
    for (int t = 0; t < T; t++) {
        for (int k = 0; k < ST_N; k++) st[k] += tst[t][k];
        free(ts[t].acc); free(ts[t].touched);
    }
    free(ts); free(tst);
    free(wprop); free(wcur); free(byid); free(stamp);
    free(volc); free(prop);
    return total;
}

/* ---------------------------------------------------------------------- */
/* coarsen (Section III-B): one coarse node per community, inter-community   */
/* weights summed, intra-community weight kept as the coarse self-loop.      */
/* pi(u) = dense rank of z[u].                                               */
/* ---------------------------------------------------------------------- */
static void coarsen(const OG *g, const int32_t *z, OG *cg, int32_t *pi)
{
    int64_t n = g->n;
    int32_t *rk = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t nc = dense_rank(n, z, rk);
    for (int64_t u = 0; u < n; u++) pi[u] = rk[z[u]];
    free(rk);
    /* members of each coarse node */
    int64_t *moff = (int64_t *)calloc((size_t)nc + 2, sizeof(int64_t));
    int32_t *mem = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    for (int64_t u = 0; u < n; u++) moff[pi[u] + 1]++;
    for (int64_t c = 0; c < nc; c++) moff[c + 1] += moff[c];
    int64_t *pos = (int64_t *)malloc(((size_t)nc + 1) * sizeof(int64_t));
    memcpy(pos, moff, (size_t)nc * sizeof(int64_t));
    for (int64_t u = 0; u < n; u++) mem[pos[pi[u]]++] = (int32_t)u;
    free(pos);

    memset(cg, 0, sizeof(*cg));
    cg->n = nc;
    cg->res_num = g->res_num;   /* every level optimises the same objective */
    cg->res_den = g->res_den;
    cg->rp = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    cg->loop = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    cg->vol = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t cap = g->rp[n] + 1;
    cg->adj = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    cg->wt = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int64_t *acc = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
    int64_t k = 0;
    for (int64_t c = 0; c < nc; c++) {
        int64_t nt = 0, intra = 0, loops = 0;
        for (int64_t i = moff[c]; i < moff[c + 1]; i++) {
            int32_t u = mem[i];
            loops += g->loop[u];
            for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
                int32_t d = pi[g->adj[e]];
                if (d == c) { intra += g->wt[e]; continue; }
                if (acc[d] == 0) touched[nt++] = d;
                acc[d] += g->wt[e];
            }
        }
        /* each intra-community edge was seen from both ends */
        cg->loop[c] = loops + intra / 2;
        /* sorted neighbour list of the coarse node */
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        for (int64_t i = 0; i < nt; i++) {
            cg->adj[k] = touched[i];
            cg->wt[k] = acc[touched[i]];
            acc[touched[i]] = 0;
            k++;
        }
        cg->rp[c + 1] = k;
    }
    free(acc); free(touched); free(moff); free(mem);
    og_volumes(cg);
}

/* ---------------------------------------------------------------------- */
/* PLM (Algorithm 3) and PLMR (Algorithm 4), recursively.                    */
/* Returns a compacted labelling of g in z (length g->n).                    */
/* ---------------------------------------------------------------------- */
typedef struct {
    uint64_t seed; int32_t max_sweeps; int32_t max_levels; int rev;
} Opts;

static void plm_rec(const OG *g, int refine, const Opts *o, int depth,
                    int32_t *z, int64_t st[ST_N])
{
    int64_t n = g->n;
    if (depth + 1 > st[ST_LEVELS]) st[ST_LEVELS] = depth + 1;
    for (int64_t u = 0; u < n; u++) z[u] = (int32_t)u;          /* singletons */
    Classes cl;
    classes_build(g, o->seed, o->rev, &cl);
    if (depth == 0) st[ST_COLORS0] = cl.ncol;
    int64_t moved = move_phase(g, z, &cl, o->seed, o->max_sweeps, st, depth == 0);
    if (moved > 0 && depth + 1 < o->max_levels) {               /* zeta changed */
        OG cg;
        int32_t *pi = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        coarsen(g, z, &cg, pi);
        int32_t *zc = (int32_t *)malloc(((size_t)cg.n + 1) * sizeof(int32_t));
        plm_rec(&cg, refine, o, depth + 1, zc, st);
        for (int64_t u = 0; u < n; u++) z[u] = zc[pi[u]];      /* prolong */
        if (refine) move_phase(g, z, &cl, o->seed, o->max_sweeps, st, depth == 0);
        free(zc); free(pi);
        og_free(&cg);
    }
    compact(n, z);
    classes_free(&cl);
}

/* ---------------------------------------------------------------------- */
/* PLP (Algorithm 1) under the colour-class schedule.                        */
/* The paper breaks ties between dominant labels arbitrarily (Section        */
/* III-A); here the tie goes to the label with the smallest                  */
/* fmix32(l ^ salt), a pseudo-random order that changes every iteration.     */
/* fmix32 is a bijection, so two labels never share a key.                   */
/* ---------------------------------------------------------------------- */
static uint32_t plp_salt(uint64_t seed, int32_t it)
{
    uint32_t s = fmix32((uint32_t)seed ^ (uint32_t)(seed >> 32));
    return fmix32(s ^ (0x9E3779B9u * (uint32_t)(it + 1)));
}

static void plp_run(const OG *g, uint64_t seed, double theta, int32_t max_iter,
                    int use_active, int rev, int32_t *z, int64_t st[ST_N])
{
    int64_t n = g->n;
    Classes cl;
    classes_build(g, seed, rev, &cl);
    st[ST_COLORS0] = cl.ncol;
    char *active = (char *)malloc((size_t)n + 1);
    char *adopt = (char *)calloc((size_t)n + 1, 1);
    int32_t *prop = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    const int T = OR_THREADS();
    Scratch *ts = (Scratch *)calloc((size_t)T, sizeof(Scratch));
    int64_t (*tst)[ST_PAD] = calloc((size_t)T, sizeof(*tst));  /* per-thread counters */
    for (int t = 0; t < T; t++) {
        ts[t].acc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        ts[t].touched = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    }
    for (int64_t v = 0; v < n; v++) { z[v] = (int32_t)v; active[v] = 1; }
    int64_t updated = n;
    int32_t it = 0;
    while ((double)updated > theta && it < max_iter) {
        updated = 0;
        uint32_t salt = plp_salt(seed, it);
        for (int32_t k = 0; k < cl.ncol; k++) {
            int64_t a = cl.off[k], b = cl.off[k + 1];
            int64_t work;
            CLASS_WORK(g, cl.v, a, b, work);
            (void)work;
            #pragma omp parallel for schedule(dynamic, 16) if (work >= OR_PAR_MIN)
            for (int64_t i = a; i < b; i++) {
                int32_t v = cl.v[i];
                Scratch *sp = &ts[OR_TID()];
                int64_t *lst = tst[OR_TID()];
                adopt[v] = 0;
                if (use_active && !active[v] && !is_hub(g, v)) continue;
                if (g->rp[v + 1] == g->rp[v]) continue;           /* deg(v) = 0 */
                int64_t nt = gather_weights(g, z, v, sp);
                int32_t bestl = -1;
                int64_t bestw = 0;
                for (int64_t j = 0; j < nt; j++) {                /* dominant label */
                    int32_t l = sp->touched[j];
                    if (bestl < 0 || sp->acc[l] > bestw ||
                        (sp->acc[l] == bestw && fmix32((uint32_t)l ^ salt) < fmix32((uint32_t)bestl ^ salt))) {
                        bestl = l; bestw = sp->acc[l];
                    }
                }
                int64_t wcur = sp->acc[z[v]];
                lst[ST_ENTRIES] += g->rp[v + 1] - g->rp[v];
                lst[ST_CANDIDATES] += nt;
                lst[ST_DECISIONS] += 1;
                clear_weights(sp, nt);
                if (bestw > wcur) { adopt[v] = 1; prop[v] = bestl; }
                else adopt[v] = 2;
            }
            for (int64_t i = a; i < b; i++) {
                int32_t v = cl.v[i];
                if (adopt[v] == 1) {
                    z[v] = prop[v];
                    updated++;
                    for (int64_t e = g->rp[v]; e < g->rp[v + 1]; e++) active[g->adj[e]] = 1;
                } else if (adopt[v] == 2) {
                    active[v] = 0;
                }
            }
        }
        st[ST_MOVES] += updated;
        it++;
    }
    st[ST_ITERS] = it;
    st[ST_CONVERGED] = ((double)updated > theta) ? 0 : 1;
    for (int t = 0; t < T; t++) {
        for (int k = 0; k < ST_N; k++) st[k] += tst[t][k];
        free(ts[t].acc); free(ts[t].touched);
    }
    free(ts); free(tst);
    compact(n, z);
    classes_free(&cl);
    free(active); free(adopt); free(prop);
}

/* ---------------------------------------------------------------------- */
/* combine (Section III-D, Eq. (2)): u and v share a core community iff     */
/* they share a community in every base solution.  Folded pairwise: the     */
/* running core id and the next base label form a 64-bit key; keys are      */
/* replaced by their dense rank.                                            */
/* ---------------------------------------------------------------------- */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int64_t combine(int64_t n, int b, const int32_t *labels, int32_t *core)
{
    for (int64_t v = 0; v < n; v++) core[v] = labels[v];
    int64_t k = compact(n, core);
    uint64_t *key = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t *srt = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    for (int i = 1; i < b; i++) {
        const int32_t *zi = labels + (size_t)i * n;
        for (int64_t v = 0; v < n; v++) key[v] = ((uint64_t)(uint32_t)core[v] << 32) | (uint32_t)zi[v];
        memcpy(srt, key, (size_t)n * sizeof(uint64_t));
        qsort(srt, (size_t)n, sizeof(uint64_t), cmp_u64);
        int64_t nu = 0;
        for (int64_t j = 0; j < n; j++) if (j == 0 || srt[j] != srt[j - 1]) srt[nu++] = srt[j];
        for (int64_t v = 0; v < n; v++) {                       /* rank by binary search */
            int64_t lo = 0, hi = nu - 1;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (srt[mid] < key[v]) lo = mid + 1; else hi = mid; }
            core[v] = (int32_t)lo;
        }
        k = nu;
    }
    free(key); free(srt);
    return k;
}

/* ====================================================================== */
/* Exported entry points (called through ctypes by the test suite).        */
/* Input CSR: row_ptr int64[n+1], col int32[nnz] (symmetric, self-loop once */
/* in its row), w int64[nnz] or NULL for unit weights.  Labels in [0, n).  */
/* Return 0 on success, -1 on allocation failure.                          */
/* ====================================================================== */

static void put128(i128 x, int64_t *out)
{
    out[0] = (int64_t)(x >> 64);
    out[1] = (int64_t)(uint64_t)x;
}

/* modularity; num_den (optional) receives N and D as (hi, lo) int64 pairs */
int or_modularity(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                  const int32_t *labels, double *mod, int64_t *num_den)
{
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    i128 N = 0, D = 0;
    if (n > 0) og_mod_num(&g, labels, &N, &D);
    *mod = og_modularity(&g, labels);
    if (num_den) { put128(N, num_den); put128(D, num_den + 2); }
    og_free(&g);
    return 0;
}

/* gain numerator g (x 2W^2) of moving u from labels[u] to community D */
int or_gain(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
            const int32_t *labels, int32_t u, int32_t D, int64_t res_num, int64_t res_den, int64_t *g_out)
{
    OG g;
    if (res_num < 0 || res_den < 1) return -2;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    if (og_set_resolution(&g, res_num, res_den)) { og_free(&g); return -2; }
    int64_t *volc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t x = 0; x < n; x++) volc[labels[x]] += g.vol[x];
    int64_t wD = 0, wC = 0;
    for (int64_t e = g.rp[u]; e < g.rp[u + 1]; e++) {
        if (labels[g.adj[e]] == D) wD += g.wt[e];
        if (labels[g.adj[e]] == labels[u]) wC += g.wt[e];
    }
    put128(gain(&g, wD, wC, g.vol[u], volc[D], volc[labels[u]]), g_out);
    free(volc);
    og_free(&g);
    return 0;
}

/* threads of the OpenMP build (no effect in the plain build); returns the
 * number the next parallel class will use */
int or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
    return OR_THREADS();
}

/* the schedule's colouring (greedy in descending priority order) */
int32_t or_color(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                 uint64_t seed, int32_t *color)
{
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    int32_t k = n ? color_greedy(&g, seed, color) : 0;
    og_free(&g);
    return k;
}

/* the same colouring by Jones-Plassmann rounds (small graphs: it rescans
 * every uncoloured vertex in every round) */
int32_t or_color_jp(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                    uint64_t seed, int32_t *color)
{
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    int32_t k = n ? color_jp(&g, seed, color) : 0;
    og_free(&g);
    return k;
}

/* one move phase at the input level, starting from labels (in/out) */
int or_move_phase(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                  uint64_t seed, int32_t max_sweeps, int rev, int32_t *labels, int64_t *stats)
{
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    int64_t st[ST_N] = {0};
    st[ST_CONVERGED] = 1;
    Classes cl;
    classes_build(&g, seed, rev, &cl);
    st[ST_COLORS0] = cl.ncol;
    move_phase(&g, labels, &cl, seed, max_sweeps, st, 1);
    classes_free(&cl);
    og_free(&g);
    memcpy(stats, st, sizeof(st));
    return 0;
}

int or_plm(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
           int refine, uint64_t seed, int32_t max_sweeps, int32_t max_levels, int rev,
           int64_t res_num, int64_t res_den, int32_t *labels, double *mod, int64_t *stats)
{
    OG g;
    if (res_num < 0 || res_den < 1) return -2;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    if (og_set_resolution(&g, res_num, res_den)) { og_free(&g); return -2; }
    int64_t st[ST_N] = {0};
    st[ST_CONVERGED] = 1;
    Opts o = { seed, max_sweeps, max_levels, rev };
    if (n > 0) plm_rec(&g, refine, &o, 0, labels, st);
    *mod = og_modularity(&g, labels);
    int64_t k = 0;
    for (int64_t u = 0; u < n; u++) if (labels[u] + 1 > k) k = labels[u] + 1;
    st[ST_NCOMM] = k;
    memcpy(stats, st, sizeof(st));
    og_free(&g);
    return 0;
}

int or_plp(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
           uint64_t seed, double theta, int32_t max_iter, int use_active, int rev,
           int32_t *labels, double *mod, int64_t *stats)
{
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    int64_t st[ST_N] = {0};
    if (n > 0) plp_run(&g, seed, theta, max_iter, use_active, rev, labels, st);
    else st[ST_CONVERGED] = 1;
    *mod = og_modularity(&g, labels);
    int64_t k = 0;
    for (int64_t u = 0; u < n; u++) if (labels[u] + 1 > k) k = labels[u] + 1;
    st[ST_NCOMM] = k;
    memcpy(stats, st, sizeof(st));
    og_free(&g);
    return 0;
}

int64_t or_combine(int64_t n, int b, const int32_t *labels, int32_t *core)
{
    return combine(n, b, labels, core);
}

/* Coarse graph of (input graph, labels) in input-CSR form (self-loop once
 * in its row).  Output buffers: rp_out [n+1], col_out / w_out [nnz + n],
 * pi_out [n].  Returns the number of coarse nodes. */
int64_t or_coarsen(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                   const int32_t *labels, int64_t *rp_out, int32_t *col_out,
                   int64_t *w_out, int32_t *pi_out)
{
    OG g, cg;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    coarsen(&g, labels, &cg, pi_out);
    int64_t k = 0;
    rp_out[0] = 0;
    for (int64_t c = 0; c < cg.n; c++) {
        int loop_done = 0;
        for (int64_t e = cg.rp[c]; e <= cg.rp[c + 1]; e++) {
            int32_t d = e < cg.rp[c + 1] ? cg.adj[e] : INT32_MAX;
            if (!loop_done && cg.loop[c] > 0 && d > c) {
                col_out[k] = (int32_t)c; w_out[k] = cg.loop[c]; k++;
                loop_done = 1;
            }
            if (e < cg.rp[c + 1]) { col_out[k] = d; w_out[k] = cg.wt[e]; k++; }
        }
        rp_out[c + 1] = k;
    }
    int64_t nc = cg.n;
    og_free(&g); og_free(&cg);
    return nc;
}

/* EPP (Algorithm 5): b PLP base runs (seed + i), exact core communities,
 * coarsen, final PLM or PLMR (final_refine) on the core graph, prolong.
 * The final phase optimises the resolution res_num / res_den (PLP has none).
 * base_out [b*n] and core_out [n] are optional. */
int or_epp(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
           int b, int final_refine, uint64_t seed, int32_t max_sweeps, int32_t max_levels,
           double theta, int32_t max_iter, int64_t res_num, int64_t res_den,
           int32_t *labels, int32_t *base_out, int32_t *core_out, double *mod, int64_t *stats)
{
    OG g;
    if (res_num < 0 || res_den < 1) return -2;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    if (og_set_resolution(&g, res_num, res_den)) { og_free(&g); return -2; }
    int64_t st[ST_N] = {0};
    st[ST_CONVERGED] = 1;
    int32_t *base = (int32_t *)malloc(((size_t)b * n + 1) * sizeof(int32_t));
    int32_t *core = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    for (int i = 0; i < b; i++) {
        int64_t sb[ST_N] = {0};
        plp_run(&g, seed + (uint64_t)i, theta, max_iter, 1, 0, base + (size_t)i * n, sb);
        st[ST_ITERS] += sb[ST_ITERS];
    }
    if (n > 0) combine(n, b, base, core);
    OG cg;
    int32_t *pi = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    coarsen(&g, core, &cg, pi);
    int32_t *zc = (int32_t *)malloc(((size_t)cg.n + 1) * sizeof(int32_t));
    Opts o = { seed, max_sweeps, max_levels, 0 };
    if (cg.n > 0) plm_rec(&cg, final_refine, &o, 0, zc, st);
    for (int64_t u = 0; u < n; u++) labels[u] = zc[pi[u]];          /* prolong */
    compact(n, labels);
    *mod = og_modularity(&g, labels);
    int64_t k = 0;
    for (int64_t u = 0; u < n; u++) if (labels[u] + 1 > k) k = labels[u] + 1;
    st[ST_NCOMM] = k;
    if (base_out) memcpy(base_out, base, (size_t)b * n * sizeof(int32_t));
    if (core_out) memcpy(core_out, core, (size_t)n * sizeof(int32_t));
    memcpy(stats, st, sizeof(st));
    free(base); free(core); free(pi); free(zc);
    og_free(&cg); og_free(&g);
    return 0;
}

/* Generic EPP(b, Base, Final) (Section III-D: the scheme is agnostic to its
 * base and final algorithms) with iterated ensembles (the hierarchy of core
 * graphs that Section II describes for the scheme EPP adapts).
 *   base: 0 PLP, 1 PLM, 2 PLMR; final: PLM, or PLMR when final_refine.
 *   Round r = 0, 1, ... < rounds: b base runs on the current graph (seeds
 *   seed + r b + i), their exact core communities (Eq. 2).  Round 0's core
 *   is always taken (Algorithm 5).  A later round's core is taken only if it
 *   merges vertices of the current graph and its modularity is strictly
 *   higher than the previous core's (quality must improve); else the rounds
 *   stop.  A taken core coarsens the current graph.  The final algorithm runs
 *   on the last graph (seed), and its labels are prolonged back through
 *   every core graph and compacted.  rounds = 1 with PLP bases is or_epp.
 * The final phase optimises the resolution res_num / res_den. */
int or_epp_general(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                   int b, int base, int final_refine, int rounds, uint64_t seed,
                   int32_t max_sweeps, int32_t max_levels, double theta, int32_t max_iter,
                   int64_t res_num, int64_t res_den, int32_t *labels, double *mod, int64_t *stats)
{
    if (b < 1 || base < 0 || base > 2 || rounds < 1 || rounds > 64) return -2;
    if (res_num < 0 || res_den < 1) return -2;
    OG g;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    if (og_set_resolution(&g, res_num, res_den)) { og_free(&g); return -2; }
    int64_t st[ST_N] = {0};
    st[ST_CONVERGED] = 1;
    OG lv[64];                 /* taken core graphs */
    int32_t *pi[64];           /* pi[l]: vertex of level l -> vertex of lv[l] (level 0 = g) */
    int nl = 0;
    const OG *cur = &g;
    double prev = 0.0;
    for (int r = 0; r < rounds; r++) {
        const int64_t nc = cur->n;
        int32_t *bl = (int32_t *)malloc(((size_t)b * nc + 1) * sizeof(int32_t));
        int32_t *core = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
        for (int i = 0; i < b; i++) {
            const uint64_t sd = seed + (uint64_t)r * (uint64_t)b + (uint64_t)i;
            int64_t sb[ST_N] = {0};
            sb[ST_CONVERGED] = 1;
            int32_t *zi = bl + (size_t)i * nc;
            if (base == 0) {
                if (nc > 0) plp_run(cur, sd, theta, max_iter, 1, 0, zi, sb);
            } else {
                Opts ob = { sd, max_sweeps, max_levels, 0 };
                if (nc > 0) plm_rec(cur, base == 2, &ob, 0, zi, sb);
            }
            st[ST_ITERS] += sb[ST_ITERS];
        }
        const int64_t k = nc > 0 ? combine(nc, b, bl, core) : 0;
        const double q = og_modularity(cur, core);
        if (r > 0 && (k == nc || q <= prev)) {      /* no contraction or no gain */
            free(bl); free(core);
            break;
        }
        prev = q;
        pi[nl] = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
        coarsen(cur, core, &lv[nl], pi[nl]);
        cur = &lv[nl];
        nl++;
        free(bl); free(core);
    }
    int32_t *z = (int32_t *)malloc(((size_t)cur->n + 1) * sizeof(int32_t));
    Opts o = { seed, max_sweeps, max_levels, 0 };
    if (cur->n > 0) plm_rec(cur, final_refine, &o, 0, z, st);
    for (int l = nl - 1; l >= 0; l--) {            /* prolong */
        const int64_t nb = l == 0 ? g.n : lv[l - 1].n;
        int32_t *zb = (int32_t *)malloc(((size_t)nb + 1) * sizeof(int32_t));
        for (int64_t v = 0; v < nb; v++) zb[v] = z[pi[l][v]];
        free(z);
        z = zb;
    }
    for (int64_t v = 0; v < n; v++) labels[v] = z[v];
    compact(n, labels);
    *mod = og_modularity(&g, labels);
    int64_t k = 0;
    for (int64_t u = 0; u < n; u++) if (labels[u] + 1 > k) k = labels[u] + 1;
    st[ST_NCOMM] = k;
    st[ST_LEVELS] = nl;        /* core graphs taken (ensemble rounds) */
    memcpy(stats, st, sizeof(st));
    free(z);
    for (int l = 0; l < nl; l++) { og_free(&lv[l]); free(pi[l]); }
    og_free(&g);
    return 0;
}

/* Number of vertices that have a neighbour community with positive gain
 * under `labels` (the convergence condition of Algorithm 2) for the
 * resolution res_num / res_den; the largest such gain numerator goes to
 * max_gain as (hi, lo).  -2: invalid resolution. */
int64_t or_positive_moves(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                          const int32_t *labels, int64_t res_num, int64_t res_den,
                          int64_t *max_gain)
{
    OG g;
    if (res_num < 0 || res_den < 1) return -2;
    if (og_from_input(&g, n, rp, col, w)) return -1;
    if (og_set_resolution(&g, res_num, res_den)) { og_free(&g); return -2; }
    int64_t *volc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t x = 0; x < n; x++) volc[labels[x]] += g.vol[x];
    Scratch s;
    s.acc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s.touched = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t cnt = 0;
    i128 mx = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t nt = gather_weights(&g, labels, u, &s);
        int32_t C = labels[u];
        for (int64_t i = 0; i < nt; i++) {
            int32_t D = s.touched[i];
            if (D == C) continue;
            i128 gD = gain(&g, s.acc[D], s.acc[C], g.vol[u], volc[D], volc[C]);
            if (gD > 0) { cnt++; if (gD > mx) mx = gD; break; }
        }
        clear_weights(&s, nt);
    }
    if (max_gain) put128(mx, max_gain);
    free(volc); free(s.acc); free(s.touched);
    og_free(&g);
    return cnt;
}
