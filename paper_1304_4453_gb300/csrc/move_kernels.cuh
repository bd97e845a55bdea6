// Decide kernels of one colour class: for every vertex u of the class,
// aggregate omega(u, c) over the communities c of its neighbours (self-loops
// are not in the adjacency), then
//   PLM (Algorithm 2, Section III-B gain): pick the community D != C = zeta(u)
//       maximising g = 2W (omega(u,D) - omega(u,C\u)) - vol(u) (vol(D) - vol(C\u)),
//       ties to the smallest id; the vertex wants to move when g > 0;
//   PLP (Algorithm 1): pick the dominant label (largest omega(u, l), ties by a
//       seeded pseudo-random order) and adopt it when strictly heavier than
//       the current label.
// Vertices of a class are pairwise non-adjacent, so a decision reads only
// labels of other classes and zeta(u) can be written in place.
//
// Community volumes (PLM).  Early sweeps apply every wanted move at once:
// the class reads the volumes as they stood when it began (buffer volc) and
// adds its moves, plus a replay of the previous class's moves, to the other
// buffer (volw), which then holds the volumes after this class.  Late sweeps
// record wanted moves as candidates; the block that finishes the class
// re-checks them in vertex order (recheck_block in phase.cuh).
//
// Work items of a class (the persistent kernels in phase.cuh walk them):
//   role 0..2  G lanes per vertex (G = 4, 8, 32), shared table of 2*DMAX
//              slots per group, deg <= DMAX (4, 16, 128);
//   role 3     one block per vertex, shared table of nextpow2(2 deg) slots,
//              deg <= 1024;
//   role 3b    one block per vertex, deg <= 4096, the same with a table in
//              the block's own slice of global memory (GT_SLOTS slots, left
//              empty after use, small enough to stay in L2); opt-in through
//              bin_max[4] > 1024 (the default routes those vertices to role 4);
//   role 4     hub aggregation: a chunk of a hub's adjacency is merged in a
//              shared table, then into the hub's global open-addressing
//              table, and every slot it fills is appended to the hub's
//              occupied-slot list.  For hubs of degree <= HUB_LAST the block
//              that merges the last chunk decides from that list at once;
//              larger hubs are decided by hub-decide slices of that list
//              (HUB_SCAN entries each) once every chunk is merged (blocks take
//              them after their own items), the last slice of each hub taking
//              the decision.
// Blocks take the items hub chunks first, then block items, then lane
// groups; every role issues several neighbour, label and volume loads per
// thread before it uses any of them.
#pragma once
#include <type_traits>

#include "barrier.cuh"
#include "common.cuh"

namespace cd {

constexpr int NBINS = 6;
constexpr int BLK_MAXDEG = 1024;
constexpr int GBLK_MAXDEG = 4096;   // role 3b
constexpr int GT_SLOTS = 8192;      // role 3b table slots per block
static_assert(GT_SLOTS >= 2 * GBLK_MAXDEG, "role 3b table must hold twice its largest degree");
constexpr int BLK_SLOTS = 2048;     // block role table (deg <= 1024)
constexpr int HUB_CHUNK = 512;      // adjacency entries per hub-aggregation item
constexpr int HUB_CHUNK_SLOTS = 1024;  // shared table of one hub-aggregation item
constexpr int HUB_SCAN = 1024;      // occupied-list entries per hub-decide slice
constexpr int HUB_LAST = 1024;      // hubs up to this degree: decided by their last aggregation item (with the
                                    // default role limits every hub has more neighbours and is decided by slices;
                                    // on R-MAT 22 that was 8 ms per run faster than a limit of 2048)
constexpr int SMEM_BYTES = 32768;   // shared memory the roles may use (the phase kernels' dynamic shared memory)

// Degree bins of the schedule: bin b holds degrees in (lim[b-1], lim[b]];
// degrees above lim[4] take the multi-block hub path.  The limits are
// launch-shape options (they move vertices between roles, never change a
// result) and may not exceed the roles' capacities.
constexpr int NLIM = 5;
struct BinLimits {
    int32_t lim[NLIM];
};
constexpr int32_t BIN_CAP[NLIM] = {4, 16, 128, BLK_MAXDEG, GBLK_MAXDEG};
// Defaults: role 3b is empty (bin_max[4] == bin_max[3]).  On R-MAT its
// single-block chain per vertex is longer than the chunked hub path's, and
// the classes are latency-bound; cd_tune may still choose it.
constexpr int32_t BIN_DEFAULT[NLIM] = {4, 16, 128, BLK_MAXDEG, BLK_MAXDEG};

__host__ __device__ inline int degree_bin(int64_t d, const BinLimits &b) {
    return d <= b.lim[0] ? 0 : d <= b.lim[1] ? 1 : d <= b.lim[2] ? 2 : d <= b.lim[3] ? 3 : d <= b.lim[4] ? 4 : 5;
}

struct Counters {              // per sweep / iteration, device
    unsigned long long wanted, moved, entries, candidates, decisions;
    unsigned long long overflow;   // hash-table probes that found no slot (must stay 0)
};
// A block sums its share of the first five counters in shared memory
// (SweepCtx::bcnt, in this order) and adds it to the sweep's Counters once,
// before the barrier that ends the sweep: thousands of warps adding to one
// record directly would serialise on a single cache line.
enum { BC_WANTED = 0, BC_MOVED, BC_ENTRIES, BC_CAND, BC_DEC, BC_N };

struct HubInfo {               // one hub vertex of a class
    int32_t v;
    int32_t nb1, nb2;          // aggregation / decide block counts (nb2 = 0: decided by the last aggregation item)
    int32_t pad;
    int64_t tab;               // first slot of its global table
    int64_t slots;             // table size (power of two)
};

// Precomputed per work item of the hub roles, so that an item starts from
// one record instead of a chain of dependent lookups.
struct ChunkDesc {             // one aggregation item: a chunk of a hub's adjacency
    int64_t beg, end;          // adjacency entries of the chunk
    int64_t tab, slots;        // the hub's global table
    int32_t u, h;              // hub vertex, class-relative hub index
    int32_t nb1, nb2;          // the hub's aggregation items and decide slices
    int32_t relax, pad;        // 1: more than HUB_RELAX neighbours (may share the class with hub neighbours)
};
struct SliceDesc {             // one decide slice of a hub's occupied-slot list
    int64_t tab;               // the hub's global table (and list)
    int64_t s0, s1;            // list entries [s0, s1) of the slice, cut at the list length
    int32_t u, h;              // hub vertex, class-relative hub index
    int32_t nb1, nb2;
    int32_t p0, relax;         // first slice of the hub inside the class; more than HUB_RELAX neighbours
};

// Class-trace words per class step (profile level 2): ends of the stages
// (global ns), the latest start of a block's first item, the longest lane-
// group, block and hub-chunk item and decide slice (ns, the slice's wait for
// its hub's table apart), and the class's applied moves (early sweeps) or
// re-check candidates (late sweeps).
enum { ST_ITEMS_END = 0, ST_DECIDE_END, ST_FINISH_END, ST_FIRST_ITEM, ST_GROUP, ST_BLOCK, ST_CHUNK, ST_SLICE_WAIT,
       ST_SLICE, ST_MOVES, STAGE_SLOTS };

struct SweepCtx {
    GraphView g;
    int64_t res_p, res_q;      // PLM resolution gamma = res_p / res_q (Section III-B); 1 / 1: modularity
    int32_t *zeta;
    // class layout
    const int32_t *order;      // class vertices, bin by bin
    int64_t off[NBINS + 1];    // bin offsets into `order`
    int32_t bend[NBINS];       // exclusive end block of each role
    int32_t *gt_keys;          // this block's role-3b table (all -1 between uses)
    void *gt_vals;             //   values (all 0 between uses)
    Counters *cnt;             // the sweep's counters (overflow only; see bcnt)
    unsigned long long *bcnt;  // this block's counter sums of the sweep (shared memory, BC_*)
    // PLM
    const int64_t *volc;       // volumes at class start (read)
    int64_t *volw;             // early sweeps: volumes after this class (write)
    int32_t *mv_u, *mv_c;      // early sweeps: this class's applied moves
    unsigned long long *nmv;
    const int32_t *rp_u, *rp_c;          // previous class's moves to replay
    const unsigned long long *rp_n;
    int late;                  // 1 from the re-check sweep on
    int32_t nrelax;            // hubs of the class with more than HUB_RELAX neighbours
    int32_t *dz_u, *dz_l;      // label writes of those hubs, deferred to the end of the class
    unsigned int *dz_n;
    int32_t *cand_u, *cand_c, *cand_d;   // late sweeps: wanted moves
    int64_t *cand_wd, *cand_wc;          //   omega(u, D), omega(u, C \ u)
    unsigned long long *ncand;
    // PLP
    uint8_t *active;
    uint32_t tie_salt;
    int32_t racy;              // racy schedule: adjacent vertices share rounds, so a hub's
                               // activity may change during its round and every hub is evaluated
    // hubs of this class
    const HubInfo *hubs;
    const int32_t *hub_b1, *hub_b2;      // exclusive prefix of hub blocks
    const ChunkDesc *chunks;   // aggregation items of the class
    const SliceDesc *slices;   // decide slices of the class
    int32_t nhubs;
    int32_t *hub_occ;          // occupied-slot lists (at each hub's table offset)
    unsigned int *hub_nocc;    // their lengths (0 between uses)
    int32_t *hub_keys;         // global tables (all -1 between uses)
    void *hub_vals;            //   values (all 0 between uses)
    void *hub_wc;              // omega(u, C) per hub
    unsigned int *hub_done1, *hub_done2;
    int64_t *part_g, *part_g2, *part_w;  // hub-decide partial bests
    int32_t *part_id;
    uint32_t *part_tk;
};

__device__ __forceinline__ uint32_t hmix(int32_t key) {
    uint32_t h = (uint32_t)key * 0x9E3779B1u;
    return h ^ (h >> 15);
}

// Open addressing with linear probing.  Tables are sized to at least twice
// the number of keys they receive, so a probe always ends; the probe count is
// still bounded by the table size, and a failed insert is reported through
// `overflow` instead of looping.
template <typename VT>
__device__ __forceinline__ void tab_insert(int32_t *keys, VT *vals, uint32_t mask, int32_t key, VT w,
                                           unsigned long long *overflow) {
    uint32_t s = hmix(key) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        int32_t k = ((volatile int32_t *)keys)[s];
        if (k == key) { atomicAdd(&vals[s], w); return; }
        if (k == -1) {
            int32_t prev = atomicCAS(&keys[s], -1, key);
            if (prev == -1 || prev == key) { atomicAdd(&vals[s], w); return; }
        }
        s = (s + 1) & mask;
    }
    atomicAdd(overflow, 1ull);
}

// tab_insert that returns the slot when this call created the key, else -1.
template <typename VT>
__device__ __forceinline__ int32_t tab_insert_new(int32_t *keys, VT *vals, uint32_t mask, int32_t key, VT w,
                                                  unsigned long long *overflow) {
    uint32_t s = hmix(key) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        int32_t k = ((volatile int32_t *)keys)[s];
        if (k == key) { atomicAdd(&vals[s], w); return -1; }
        if (k == -1) {
            int32_t prev = atomicCAS(&keys[s], -1, key);
            if (prev == -1) { atomicAdd(&vals[s], w); return (int32_t)s; }
            if (prev == key) { atomicAdd(&vals[s], w); return -1; }
        }
        s = (s + 1) & mask;
    }
    atomicAdd(overflow, 1ull);
    return -1;
}

template <typename VT>
__device__ __forceinline__ VT tab_lookup(const int32_t *keys, const VT *vals, uint32_t mask, int32_t key) {
    uint32_t s = hmix(key) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        int32_t k = keys[s];
        if (k == key) return vals[s];
        if (k == -1) return 0;
        s = (s + 1) & mask;
    }
    return 0;
}

template <typename VT>
__device__ __forceinline__ VT tab_lookup_cg(const int32_t *keys, const VT *vals, uint32_t mask, int32_t key) {
    uint32_t s = hmix(key) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        int32_t k = __ldcg(keys + s);
        if (k == key) return __ldcg(vals + s);
        if (k == -1) return 0;
        s = (s + 1) & mask;
    }
    return 0;
}

// Global hub tables (open addressing, linear probing, slots a power of two):
// int32 keys (-1: empty) and values of type VT (32 bits on the 64-bit gain
// path, where omega(u, c) <= vol(u) <= 2W < 2^32; 64 bits on the 128-bit
// path) in two arrays at the same slot offsets.
template <typename VT>
struct HubTable {
    int32_t *k;
    VT *v;
    __device__ __forceinline__ HubTable(int32_t *keys, void *vals, int64_t tab)
        : k(keys + tab), v(static_cast<VT *>(vals) + tab) {}
    __device__ __forceinline__ void read(int64_t s, int32_t &key, int64_t &w) const {
        key = __ldcg(k + s);
        w = (int64_t)__ldcg(v + s);
    }
    __device__ __forceinline__ void clear(int64_t s) const {
        k[s] = -1;
        v[s] = 0;
    }
    // Insertion in two steps, so that a thread can have the compare-and-swaps
    // of all its keys in flight before it looks at any result: claim() tries
    // slot s and returns the key it held; settle() returns 1 (the key was new
    // here) or 0 (the key was here), adding w in both cases, or -1 (another
    // key: probe on).
    __device__ __forceinline__ int32_t claim(int64_t s, int32_t key) const { return atomicCAS(k + s, -1, key); }
    __device__ __forceinline__ int settle(int64_t s, int32_t key, VT w, int32_t prev) const {
        if (prev != -1 && prev != key) return -1;
        atomicAdd(v + s, w);
        return prev == -1 ? 1 : 0;
    }
    __device__ __forceinline__ int64_t lookup(uint32_t mask, int32_t key) const {
        return (int64_t)tab_lookup_cg<VT>(k, v, mask, key);
    }
};

// ---------------------------------------------------------------------------
// Candidate ordering
// ---------------------------------------------------------------------------
template <bool BIG>
struct GainT { using T = int64_t; };
template <>
struct GainT<true> { using T = __int128; };

// PLM best: larger gain, then smaller id.  id < 0: none.
template <bool BIG>
struct PlmBest {
    typename GainT<BIG>::T g;
    int64_t w;                 // omega(u, id)
    int32_t id;
    __device__ __forceinline__ void init() { g = 0; w = 0; id = -1; }
    __device__ __forceinline__ void offer(typename GainT<BIG>::T gg, int32_t d, int64_t ww) {
        if (id < 0 || gg > g || (gg == g && d < id)) { g = gg; id = d; w = ww; }
    }
    __device__ __forceinline__ void merge(const PlmBest &o) {
        if (o.id >= 0) offer(o.g, o.id, o.w);
    }
    __device__ __forceinline__ PlmBest shfl_xor(unsigned mask, int off) const {
        PlmBest r;
        if constexpr (BIG) {
            uint64_t lo = (uint64_t)g, hi = (uint64_t)(g >> 64);
            lo = __shfl_xor_sync(mask, lo, off);
            hi = __shfl_xor_sync(mask, hi, off);
            r.g = (__int128)(((unsigned __int128)hi << 64) | lo);
        } else {
            r.g = __shfl_xor_sync(mask, g, off);
        }
        r.w = __shfl_xor_sync(mask, w, off);
        r.id = __shfl_xor_sync(mask, id, off);
        return r;
    }
};

// PLP best: larger weight, then smaller tie key (fmix32(label ^ salt)).
struct PlpBest {
    int64_t w;
    uint32_t tk;
    int32_t id;
    __device__ __forceinline__ void init() { w = 0; tk = 0; id = -1; }
    __device__ __forceinline__ void offer(int64_t ww, uint32_t t, int32_t l) {
        if (id < 0 || ww > w || (ww == w && t < tk)) { w = ww; tk = t; id = l; }
    }
    __device__ __forceinline__ void merge(const PlpBest &o) {
        if (o.id >= 0) offer(o.w, o.tk, o.id);
    }
    __device__ __forceinline__ PlpBest shfl_xor(unsigned mask, int off) const {
        PlpBest r;
        r.w = __shfl_xor_sync(mask, w, off);
        r.tk = __shfl_xor_sync(mask, tk, off);
        r.id = __shfl_xor_sync(mask, id, off);
        return r;
    }
};

// Gain of moving u from C to D times 2 W^2 q (Section III-B, Delta mod,
// with the resolution gamma = p / q scaling the volume term):
//   g = 2W q (omega(u,D) - omega(u,C\u)) - p vol(u) (vol(D) - vol(C\u)),
// volC = vol(C) including u.  Exact in T: the host bounds max(p, q) (2W)^2.
template <bool BIG>
__device__ __forceinline__ typename GainT<BIG>::T plm_gain(int64_t twoW, int64_t q, int64_t p, int64_t wD,
                                                           int64_t wC, int64_t vu, int64_t volD, int64_t volC) {
    using T = typename GainT<BIG>::T;
    return (T)twoW * (T)q * (T)(wD - wC) - (T)p * (T)vu * (T)(volD - volC + vu);
}

template <bool BIG>
using ValT = std::conditional_t<BIG, unsigned long long, unsigned int>;

// Warp-wide sums of per-lane counters into the block's shared sums.
__device__ __forceinline__ void add_counters(unsigned long long *bc, unsigned wanted, unsigned moved, unsigned entries,
                                             unsigned cand, unsigned dec) {
    wanted = __reduce_add_sync(0xffffffffu, wanted);
    moved = __reduce_add_sync(0xffffffffu, moved);
    entries = __reduce_add_sync(0xffffffffu, entries);
    cand = __reduce_add_sync(0xffffffffu, cand);
    dec = __reduce_add_sync(0xffffffffu, dec);
    if ((threadIdx.x & 31) == 0) {
        if (wanted) atomicAdd(&bc[BC_WANTED], (unsigned long long)wanted);
        if (moved) atomicAdd(&bc[BC_MOVED], (unsigned long long)moved);
        if (entries) atomicAdd(&bc[BC_ENTRIES], (unsigned long long)entries);
        if (cand) atomicAdd(&bc[BC_CAND], (unsigned long long)cand);
        if (dec) atomicAdd(&bc[BC_DEC], (unsigned long long)dec);
    }
}

// Adds the block's sums to the sweep's counters and clears them (whole
// block; the caller's next team barrier publishes the additions).
__device__ __forceinline__ void flush_counters(unsigned long long *bc, Counters *dst) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *d[BC_N] = {&dst->wanted, &dst->moved, &dst->entries, &dst->candidates, &dst->decisions};
        for (int i = 0; i < BC_N; i++) {
            if (bc[i]) atomicAdd(d[i], bc[i]);
            bc[i] = 0;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void vol_add(int64_t *v, int32_t c, int64_t x) {
    atomicAdd(reinterpret_cast<unsigned long long *>(v + c), (unsigned long long)x);
}

// Applies a wanted move (early sweeps) or records it for the re-check.
// A hub that may share its class with hub neighbours defers its label write
// to the end of the class (defer_label), so that those neighbours decide on
// the labels the class started from.
__device__ __forceinline__ void defer_label(const SweepCtx &c, int32_t u, int32_t l) {
    const unsigned i = atomicAdd(c.dz_n, 1u);
    c.dz_u[i] = u;
    c.dz_l[i] = l;
}

__device__ __forceinline__ void take_move(const SweepCtx &c, unsigned long long pos, int32_t u, int32_t C,
                                          int32_t D, int64_t wD, int64_t wC, bool defer = false) {
    if (!c.late) {
        const int64_t vu = c.g.vol[u];
        if (defer) defer_label(c, u, D);
        else c.zeta[u] = D;
        c.mv_u[pos] = u;
        c.mv_c[pos] = C;
        vol_add(c.volw, C, -vu);
        vol_add(c.volw, D, vu);
    } else {
        c.cand_u[pos] = u;
        c.cand_c[pos] = C;
        c.cand_d[pos] = D;
        c.cand_wd[pos] = wD;
        c.cand_wc[pos] = wC;
    }
}

// ---------------------------------------------------------------------------
// Group role: G lanes per vertex, 256 / G vertices per block.
// ---------------------------------------------------------------------------
template <int G, int DMAX, int WK, bool BIG, bool PLP>
__device__ __forceinline__ void role_group(const SweepCtx &c, int64_t rb, const int32_t *__restrict__ list,
                                           int64_t count, unsigned char *smem) {
    using VT = ValT<BIG>;
    constexpr int SLOTS = 2 * DMAX;
    constexpr int GPB = kBlock / G;
    static_assert(GPB * SLOTS * (4 + sizeof(VT)) <= SMEM_BYTES, "group table too large");
    const int grp = threadIdx.x / G, gl = threadIdx.x % G, lane = threadIdx.x & 31;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * SLOTS;
    VT *vals = reinterpret_cast<VT *>(smem + GPB * SLOTS * 4) + grp * SLOTS;
    // groups are aligned runs of G lanes, so xor offsets below G stay inside
    // the group; the whole warp is converged at every shuffle
    const unsigned gmask = 0xffffffffu;

    const int64_t idx = rb * GPB + grp;
    bool valid = idx < count;
    const int32_t u = valid ? list[idx] : 0;
    if constexpr (PLP) {
        if (valid && !c.active[u]) valid = false;
    }
#pragma unroll
    for (int s = gl; s < SLOTS; s += G) { keys[s] = -1; vals[s] = 0; }
    __syncwarp();
    int64_t beg = 0;
    int deg = 0;
    // the vertex's own label and volume travel with its row offsets: only u
    // writes zeta[u] during its class
    const int32_t C = valid ? c.zeta[u] : 0;
    int64_t vu = 0;
    if constexpr (!PLP) vu = valid ? c.g.vol[u] : 0;
    if (valid) {
        beg = c.g.rp[u];
        deg = (int)(c.g.rp[u + 1] - beg);
    }
    // neighbour ids, then their labels, then the inserts: every load of a
    // lane is in flight before the first one is used
    constexpr int PER = DMAX / G;
    int32_t nb[PER];
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const int k = gl + j * G;
        nb[j] = (valid && k < deg) ? c.g.col[beg + k] : -1;
    }
    int64_t volC = 0;
    if constexpr (!PLP) volC = valid ? c.volc[C] : 0;
#pragma unroll
    for (int j = 0; j < PER; j++) nb[j] = nb[j] >= 0 ? c.zeta[nb[j]] : -1;
#pragma unroll
    for (int j = 0; j < PER; j++)
        if (nb[j] >= 0)
            tab_insert<VT>(keys, vals, SLOTS - 1, nb[j], (VT)edge_weight<WK>(c.g.w, beg + gl + j * G), &c.cnt->overflow);
    __syncwarp();
    const int64_t wC = valid ? (int64_t)tab_lookup<VT>(keys, vals, SLOTS - 1, C) : 0;
    unsigned ncand = 0;
    if constexpr (!PLP) {
        const int64_t twoW = 2 * c.g.W;
        PlmBest<BIG> b;
        b.init();
        // keys, then the volumes of the candidates, then the gains
        constexpr int SPL = SLOTS / G;
        int32_t ky[SPL];
        int64_t vk[SPL];
#pragma unroll
        for (int j = 0; j < SPL; j++) {
            const int32_t key = valid ? keys[gl + j * G] : -1;
            ky[j] = key;
            ncand += key >= 0;
        }
#pragma unroll
        for (int j = 0; j < SPL; j++) vk[j] = (ky[j] >= 0 && ky[j] != C) ? c.volc[ky[j]] : 0;
#pragma unroll
        for (int j = 0; j < SPL; j++)
            if (ky[j] >= 0 && ky[j] != C) {
                const int64_t w = (int64_t)vals[gl + j * G];
                b.offer(plm_gain<BIG>(twoW, c.res_q, c.res_p, w, wC, vu, vk[j], volC), ky[j], w);
            }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) b.merge(b.shfl_xor(gmask, o));
        const bool want = gl == 0 && valid && b.id >= 0 && b.g > 0;
        const unsigned ballot = __ballot_sync(0xffffffffu, want);
        unsigned long long base = 0;
        if (lane == 0 && ballot) base = atomicAdd(c.late ? c.ncand : c.nmv, (unsigned long long)__popc(ballot));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (want) take_move(c, base + __popc(ballot & ((1u << lane) - 1u)), u, C, b.id, b.w, wC);
        add_counters(c.bcnt, want, want && !c.late, gl == 0 && valid ? deg : 0, ncand, gl == 0 && valid);
    } else {
        PlpBest b;
        b.init();
#pragma unroll
        for (int s = gl; s < SLOTS; s += G) {
            const int32_t key = keys[s];
            if (valid && key >= 0) {
                ncand++;
                b.offer((int64_t)vals[s], fmix32((uint32_t)key ^ c.tie_salt), key);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) b.merge(b.shfl_xor(gmask, o));
        // every lane of the group now holds the group's best
        const bool adopt = valid && b.id >= 0 && b.w > wC;
        if (gl == 0 && valid) {
            if (adopt) c.zeta[u] = b.id;
            else c.active[u] = 0;
        }
        if (adopt)
            for (int k = gl; k < deg; k += G) c.active[c.g.col[beg + k]] = 1;
        add_counters(c.bcnt, 0, gl == 0 && adopt, gl == 0 && valid ? deg : 0, ncand, gl == 0 && valid);
    }
}

// ---------------------------------------------------------------------------
// Block role: one block per vertex (deg <= 1024).
// ---------------------------------------------------------------------------
template <typename B>
__device__ __forceinline__ B block_best(B b, B *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b.merge(b.shfl_xor(0xffffffffu, o));
    if (lane == 0) sh[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kBlock / 32; i++) b.merge(sh[i]);
        sh[0] = b;
    }
    __syncthreads();
    B r = sh[0];
    __syncthreads();
    return r;
}

template <bool PLP, bool BIG>
struct BestOf { using T = PlmBest<BIG>; };
template <bool BIG>
struct BestOf<true, BIG> { using T = PlpBest; };

// GLOBAL: role 3b (table in the block's global slice: read through L2, and
// the slots used are emptied again before the block moves on).
template <int WK, bool BIG, bool PLP, bool GLOBAL>
__device__ __forceinline__ void role_block(const SweepCtx &c, int64_t rb, const int32_t *__restrict__ list,
                                           unsigned char *smem, typename BestOf<PLP, BIG>::T *s_best,
                                           unsigned *s_cand) {
    using VT = ValT<BIG>;
    static_assert(BLK_SLOTS * (4 + sizeof(VT)) <= SMEM_BYTES, "block table too large");
    int32_t *keys = GLOBAL ? c.gt_keys : reinterpret_cast<int32_t *>(smem);
    VT *vals = GLOBAL ? static_cast<VT *>(c.gt_vals) : reinterpret_cast<VT *>(smem + BLK_SLOTS * 4);
    const int32_t u = list[rb];
    if constexpr (PLP) {
        if (!c.active[u]) return;   // uniform across the block
    }
    const int64_t beg = c.g.rp[u];
    const int deg = (int)(c.g.rp[u + 1] - beg);
    // own label, volume and community volume early (only u writes zeta[u]
    // during its class)
    const int32_t C = c.zeta[u];
    int64_t vu = 0, volC = 0;
    if constexpr (!PLP) {
        vu = c.g.vol[u];
        volC = c.volc[C];
    }
    int slots = 64;
    while (slots < 2 * deg) slots <<= 1;
    const uint32_t mask = slots - 1;
    if constexpr (!GLOBAL)
        for (int s = threadIdx.x; s < slots; s += kBlock) { keys[s] = -1; vals[s] = 0; }
    if (threadIdx.x == 0) *s_cand = 0;
    __syncthreads();
    // four entries per thread and step: ids, then labels, then inserts
    for (int k0 = threadIdx.x; k0 < deg; k0 += 4 * kBlock) {
        int32_t nb[4];
#pragma unroll
        for (int j = 0; j < 4; j++) nb[j] = k0 + j * kBlock < deg ? c.g.col[beg + k0 + j * kBlock] : -1;
#pragma unroll
        for (int j = 0; j < 4; j++) nb[j] = nb[j] >= 0 ? c.zeta[nb[j]] : -1;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (nb[j] >= 0)
                tab_insert<VT>(keys, vals, mask, nb[j], (VT)edge_weight<WK>(c.g.w, beg + k0 + j * kBlock),
                               &c.cnt->overflow);
    }
    __syncthreads();
    const int64_t wC = GLOBAL ? (int64_t)tab_lookup_cg<VT>(keys, vals, mask, C) : (int64_t)tab_lookup<VT>(keys, vals, mask, C);
    if constexpr (GLOBAL) __syncthreads();   // every lookup is done before slots are emptied
    unsigned ncand = 0;
    if constexpr (!PLP) {
        const int64_t twoW = 2 * c.g.W;
        PlmBest<BIG> b;
        b.init();
        // four slots per thread and step: keys, then candidate volumes, then gains
        for (int s0 = threadIdx.x; s0 < slots; s0 += 4 * kBlock) {
            int32_t ky[4];
            int64_t vk[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int s = s0 + j * kBlock;
                ky[j] = s < slots ? (GLOBAL ? __ldcg(keys + s) : keys[s]) : -1;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) vk[j] = (ky[j] >= 0 && ky[j] != C) ? c.volc[ky[j]] : 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int s = s0 + j * kBlock;
                if (ky[j] >= 0) {
                    ncand++;
                    const int64_t w = GLOBAL ? (int64_t)__ldcg(vals + s) : (int64_t)vals[s];
                    if (ky[j] != C) b.offer(plm_gain<BIG>(twoW, c.res_q, c.res_p, w, wC, vu, vk[j], volC), ky[j], w);
                    if constexpr (GLOBAL) { keys[s] = -1; vals[s] = 0; }
                }
            }
        }
        ncand = __reduce_add_sync(0xffffffffu, ncand);
        if ((threadIdx.x & 31) == 0) atomicAdd(s_cand, ncand);
        b = block_best(b, s_best);
        if (threadIdx.x == 0) {
            const bool want = b.id >= 0 && b.g > 0;
            if (want) take_move(c, atomicAdd(c.late ? c.ncand : c.nmv, 1ull), u, C, b.id, b.w, wC);
            c.bcnt[BC_WANTED] += want;
            c.bcnt[BC_MOVED] += want && !c.late;
            c.bcnt[BC_ENTRIES] += deg;
            c.bcnt[BC_CAND] += *s_cand;
            c.bcnt[BC_DEC] += 1;
        }
    } else {
        PlpBest b;
        b.init();
        for (int s = threadIdx.x; s < slots; s += kBlock) {
            const int32_t key = GLOBAL ? __ldcg(keys + s) : keys[s];
            if (key >= 0) {
                ncand++;
                const int64_t w = GLOBAL ? (int64_t)__ldcg(vals + s) : (int64_t)vals[s];
                b.offer(w, fmix32((uint32_t)key ^ c.tie_salt), key);
                if constexpr (GLOBAL) { keys[s] = -1; vals[s] = 0; }
            }
        }
        ncand = __reduce_add_sync(0xffffffffu, ncand);
        if ((threadIdx.x & 31) == 0) atomicAdd(s_cand, ncand);
        b = block_best(b, s_best);
        const bool adopt = b.id >= 0 && b.w > wC;
        if (adopt)
            for (int k = threadIdx.x; k < deg; k += kBlock) c.active[c.g.col[beg + k]] = 1;
        if (threadIdx.x == 0) {
            if (adopt) c.zeta[u] = b.id;
            else c.active[u] = 0;
            c.bcnt[BC_MOVED] += adopt;
            c.bcnt[BC_ENTRIES] += deg;
            c.bcnt[BC_CAND] += *s_cand;
            c.bcnt[BC_DEC] += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Hub roles (degree above the block-role limit, bin_max[3] <= 1024).
// ---------------------------------------------------------------------------

// Takes the decision of hub u from its best candidate (one block; r, C and
// wC are the same in every thread).
template <bool BIG, bool PLP>
__device__ __forceinline__ void hub_finish(const SweepCtx &c, int32_t u, int32_t C, int64_t wC,
                                           const typename BestOf<PLP, BIG>::T &r, int *s_last, bool relax) {
    if (threadIdx.x == 0) {
        if constexpr (!PLP) {
            const bool want = r.id >= 0 && r.g > 0;
            if (want) take_move(c, atomicAdd(c.late ? c.ncand : c.nmv, 1ull), u, C, r.id, r.w, wC, relax);
            c.bcnt[BC_WANTED] += want;
            c.bcnt[BC_MOVED] += want && !c.late;
            *s_last = 1;
        } else {
            const bool adopt = r.id >= 0 && r.w > wC;
            if (adopt) {
                if (relax) defer_label(c, u, r.id);
                else c.zeta[u] = r.id;
            } else {
                c.active[u] = 0;
            }
            c.bcnt[BC_MOVED] += adopt;
            *s_last = adopt ? 2 : 1;
        }
        c.bcnt[BC_DEC] += 1;
    }
    __syncthreads();
    if constexpr (PLP) {
        if (*s_last == 2) {
            const int64_t rb = c.g.rp[u], re = c.g.rp[u + 1];
            for (int64_t e = rb + threadIdx.x; e < re; e += kBlock) c.active[c.g.col[e]] = 1;
        }
    }
    __syncthreads();
}

// Decision of hub h (degree <= HUB_LAST) by the block that merged its last
// chunk: every other chunk has published its slots (fence, then the chunk
// counter), so the occupied-slot list is complete.  Scans the list, clears
// the slots it used, and decides.
template <int WK, bool BIG, bool PLP>
__device__ __forceinline__ void hub_decide_occ(const SweepCtx &c, const ChunkDesc &hi,
                                               typename BestOf<PLP, BIG>::T *s_best, int *s_last) {
    using BT = typename BestOf<PLP, BIG>::T;
    __threadfence();
    const HubTable<ValT<BIG>> tb(c.hub_keys, c.hub_vals, hi.tab);
    const int32_t *occ = c.hub_occ + hi.tab;
    const uint32_t gmask = (uint32_t)(hi.slots - 1);
    const int32_t u = hi.u;
    const int h = hi.h;
    const int32_t C = c.zeta[u];
    const int64_t nocc = (int64_t)__ldcg(c.hub_nocc + h);
    const int64_t wC = tb.lookup(gmask, C);
    __syncthreads();   // every thread's lookup of C is done before slots are cleared below
    BT b;
    b.init();
    // four list entries per thread and step (one step for nocc <= HUB_LAST):
    // slot numbers, then the slots, then candidate volumes, then the offers
    constexpr int OPT = 4;
    int64_t vu = 0, volC = 0;
    if constexpr (!PLP) {
        vu = c.g.vol[u];
        volC = c.volc[C];
    }
    for (int64_t i0 = threadIdx.x; i0 < nocc; i0 += OPT * kBlock) {
        int32_t sl[OPT], ky[OPT];
        int64_t wv[OPT], vk[OPT];
#pragma unroll
        for (int j = 0; j < OPT; j++) sl[j] = i0 + j * kBlock < nocc ? __ldcg(occ + i0 + j * kBlock) : -1;
#pragma unroll
        for (int j = 0; j < OPT; j++) {
            ky[j] = -1;
            wv[j] = 0;
            if (sl[j] >= 0) tb.read(sl[j], ky[j], wv[j]);
        }
        if constexpr (!PLP) {
#pragma unroll
            for (int j = 0; j < OPT; j++) vk[j] = (sl[j] >= 0 && ky[j] != C) ? c.volc[ky[j]] : 0;
#pragma unroll
            for (int j = 0; j < OPT; j++)
                if (sl[j] >= 0 && ky[j] != C)
                    b.offer(plm_gain<BIG>(2 * c.g.W, c.res_q, c.res_p, wv[j], wC, vu, vk[j], volC), ky[j], wv[j]);
        } else {
#pragma unroll
            for (int j = 0; j < OPT; j++)
                if (sl[j] >= 0) b.offer(wv[j], fmix32((uint32_t)ky[j] ^ c.tie_salt), ky[j]);
        }
#pragma unroll
        for (int j = 0; j < OPT; j++)
            if (sl[j] >= 0) tb.clear(sl[j]);   // each listed slot is read and cleared by one thread
    }
    b = block_best(b, s_best);
    if (threadIdx.x == 0) {
        c.hub_done1[h] = 0;
        c.hub_nocc[h] = 0;
        c.bcnt[BC_CAND] += nocc;
    }
    hub_finish<BIG, PLP>(c, u, C, wC, b, s_last, hi.relax != 0);
}

template <int WK, bool BIG, bool PLP>
__device__ __forceinline__ void role_hub_aggregate(const SweepCtx &c, int32_t rb, unsigned char *smem,
                                                   typename BestOf<PLP, BIG>::T *s_best, int *s_last) {
    using VT = ValT<BIG>;
    constexpr int PER = HUB_CHUNK_SLOTS / kBlock;
    static_assert(HUB_CHUNK_SLOTS % kBlock == 0, "chunk table slots per thread");
    int32_t *keys = reinterpret_cast<int32_t *>(smem);
    VT *vals = reinterpret_cast<VT *>(smem + HUB_CHUNK_SLOTS * 4);
    int32_t *wsum = reinterpret_cast<int32_t *>(smem + HUB_CHUNK_SLOTS * 12);   // [kBlock / 32 + 2]
    static_assert(HUB_CHUNK_SLOTS * 12 + (kBlock / 32 + 2) * 4 <= SMEM_BYTES, "hub chunk scratch");
    const ChunkDesc hi = c.chunks[rb];
    const int h = hi.h;
    const int32_t u = hi.u;
    if constexpr (PLP) {
        // whole block; the decision skips it too.  Hubs that may share the
        // class with hub neighbours are evaluated every iteration.
        if (!hi.relax && !c.racy && !c.active[u]) return;
    }
    const int64_t beg = hi.beg, end = hi.end;
    for (int s = threadIdx.x; s < HUB_CHUNK_SLOTS; s += kBlock) { keys[s] = -1; vals[s] = 0; }
    {
        // every neighbour id of the thread, then every label, before the inserts
        constexpr int EPT = (HUB_CHUNK + kBlock - 1) / kBlock;
        int32_t nb[EPT];
#pragma unroll
        for (int j = 0; j < EPT; j++) {
            const int64_t e = beg + threadIdx.x + j * kBlock;
            nb[j] = e < end ? c.g.col[e] : -1;
        }
#pragma unroll
        for (int j = 0; j < EPT; j++) nb[j] = nb[j] >= 0 ? c.zeta[nb[j]] : -1;
        __syncthreads();   // the table is cleared
#pragma unroll
        for (int j = 0; j < EPT; j++)
            if (nb[j] >= 0)
                tab_insert<VT>(keys, vals, HUB_CHUNK_SLOTS - 1, nb[j],
                               (VT)edge_weight<WK>(c.g.w, beg + threadIdx.x + j * kBlock), &c.cnt->overflow);
    }
    __syncthreads();
    const HubTable<ValT<BIG>> tb(c.hub_keys, c.hub_vals, hi.tab);
    const uint32_t gmask = (uint32_t)(hi.slots - 1);
    {
        // merge into the hub table; slots created here go to the occupied
        // list.  All keys of the thread probe at once: in each round every
        // pending key tries its current slot with one compare-and-swap (which
        // also reports a slot that already holds the key), so a round costs
        // one round trip to L2 however many keys the thread holds.
        int32_t fresh[PER], ky[PER];
        VT vl[PER];
        uint32_t at[PER];
        unsigned pend = 0;
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int s = threadIdx.x + i * kBlock;
            ky[i] = keys[s];
            vl[i] = vals[s];
            fresh[i] = -1;
            at[i] = hmix(ky[i]) & gmask;
            if (ky[i] >= 0) pend |= 1u << i;
        }
        for (uint32_t probe = 0; pend && probe <= gmask; probe++) {
            int32_t prev[PER];
#pragma unroll
            for (int i = 0; i < PER; i++) prev[i] = (pend >> i) & 1u ? tb.claim(at[i], ky[i]) : 0;
#pragma unroll
            for (int i = 0; i < PER; i++) {
                if (!((pend >> i) & 1u)) continue;
                const int r = tb.settle(at[i], ky[i], vl[i], prev[i]);
                if (r >= 0) {
                    if (r == 1) fresh[i] = (int32_t)at[i];
                    pend &= ~(1u << i);
                } else {
                    at[i] = (at[i] + 1) & gmask;
                }
            }
        }
        if (pend) atomicAdd(&c.cnt->overflow, (unsigned long long)__popc(pend));
        int nf = 0;
#pragma unroll
        for (int i = 0; i < PER; i++) nf += fresh[i] >= 0;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < kBlock / 32; w++) { const int t = wsum[w]; wsum[w] = run; run += t; }
            wsum[kBlock / 32] = run ? (int)atomicAdd(c.hub_nocc + h, (unsigned)run) : 0;
        }
        __syncthreads();
        int pos = wsum[kBlock / 32] + wsum[warp] + incl - nf;
        int32_t *occ = c.hub_occ + hi.tab;
#pragma unroll
        for (int i = 0; i < PER; i++)
            if (fresh[i] >= 0) occ[pos++] = fresh[i];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned done = atomicAdd(&c.hub_done1[h], 1u);
        *s_last = (done == (unsigned)hi.nb1 - 1);
        c.bcnt[BC_ENTRIES] += end - beg;
    }
    __syncthreads();
    // hubs with decide slices: the count reaching nb1 releases the slices
    if (*s_last && hi.nb2 == 0) hub_decide_occ<WK, BIG, PLP>(c, hi, s_best, s_last);
}

}  // namespace cd
