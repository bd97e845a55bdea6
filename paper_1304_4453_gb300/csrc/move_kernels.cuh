// Decide kernels of one colour class: for every vertex u of the class,
// aggregate omega(u, c) over the communities c of its neighbours (self-loops
// are not in the adjacency), then
//   PLM (Algorithm 2, Section III-B gain): pick the community D != C = zeta(u)
//       maximising g = 2W (omega(u,D) - omega(u,C\u)) - vol(u) (vol(D) - vol(C\u)),
//       ties to the smallest id, and move when g > 0;
//   PLP (Algorithm 1): pick the dominant label (largest omega(u, l), ties by a
//       seeded pseudo-random order) and adopt it when strictly heavier than
//       the current label.
// Vertices of a class are pairwise non-adjacent, so a decision reads only
// labels of other classes and zeta(u) can be written in place.  Community
// volumes are read from the snapshot of the class start; moves are recorded
// and applied to the volumes by k_apply_moves after the class.
//
// Aggregation by degree bin:
//   group kernels   G lanes per vertex (G = 4, 8, 32), shared table of
//                   2*DMAX slots per group, deg <= DMAX;
//   block kernel    one block per vertex, shared table of nextpow2(2 deg)
//                   slots, deg <= 1024;
//   hub kernels     several blocks per vertex: H1 pre-aggregates chunks of
//                   the adjacency in shared memory and merges them into a
//                   global open-addressing table; H2 scans slices of the
//                   table, and the last block of each hub takes the decision.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace cd {

constexpr int NBINS = 5;
constexpr int BLK_MAXDEG = 1024;
constexpr int BLK_SLOTS = 2048;     // block kernel table (deg <= 1024)
constexpr int HUB_CHUNK = 1024;     // adjacency entries per H1 block
constexpr int HUB_SCAN = 4096;      // table slots per H2 block

__host__ __device__ inline int degree_bin(int64_t d) {
    return d <= 4 ? 0 : d <= 16 ? 1 : d <= 128 ? 2 : d <= BLK_MAXDEG ? 3 : 4;
}

struct Counters {              // per sweep / iteration, device
    unsigned long long wanted, moved, entries, candidates, decisions;
};

struct HubInfo {               // one hub vertex of a class
    int32_t v;
    int32_t nb1, nb2;          // H1 / H2 block counts
    int32_t pad;
    int64_t tab;               // first slot of its global table
    int64_t slots;             // table size (power of two)
};

struct SweepCtx {
    GraphView g;
    int32_t *zeta;
    const int64_t *volc;       // PLM: community volumes at class start
    int32_t *mv_u, *mv_c;      // PLM: move records of this class
    unsigned long long *nmv;   // PLM: number of records of this class
    Counters *cnt;
    int late;                  // PLM: 1 from the re-check sweep on
    int32_t *cand_u, *cand_c, *cand_d;   // PLM late sweeps: wanted moves
    int64_t *cand_wd, *cand_wc;          //   omega(u, D), omega(u, C \ u)
    unsigned long long *ncand;           //   count for this class
    uint8_t *active;           // PLP active flags
    uint32_t tie_salt;         // PLP tie order
    // hubs of this class
    const HubInfo *hubs;
    const int32_t *hub_b1, *hub_b2;   // exclusive prefix of H1 / H2 blocks
    int32_t nhubs;
    int32_t *hub_keys;         // global tables (all -1 between uses)
    void *hub_vals;            //   values (all 0 between uses)
    void *hub_wc;              // omega(u, C) per hub (H1 -> H2)
    unsigned int *hub_done1, *hub_done2;
    int64_t *part_g;           // H2 partial bests: gain hi/lo or weight
    int64_t *part_g2;
    int64_t *part_w;           // H2 partial bests: omega(u, D) (PLM)
    int32_t *part_id;
    uint32_t *part_tk;
};

__device__ __forceinline__ uint32_t hmix(int32_t key) {
    uint32_t h = (uint32_t)key * 0x9E3779B1u;
    return h ^ (h >> 15);
}

template <typename VT>
__device__ __forceinline__ void tab_insert(int32_t *keys, VT *vals, uint32_t mask, int32_t key, VT w) {
    uint32_t s = hmix(key) & mask;
    while (true) {
        int32_t k = ((volatile int32_t *)keys)[s];
        if (k == key) { atomicAdd(&vals[s], w); return; }
        if (k == -1) {
            int32_t prev = atomicCAS(&keys[s], -1, key);
            if (prev == -1 || prev == key) { atomicAdd(&vals[s], w); return; }
        }
        s = (s + 1) & mask;
    }
}

template <typename VT>
__device__ __forceinline__ VT tab_lookup(const int32_t *keys, const VT *vals, uint32_t mask, int32_t key) {
    uint32_t s = hmix(key) & mask;
    while (true) {
        int32_t k = keys[s];
        if (k == key) return vals[s];
        if (k == -1) return 0;
        s = (s + 1) & mask;
    }
}

template <typename VT>
__device__ __forceinline__ VT tab_lookup_cg(const int32_t *keys, const VT *vals, uint32_t mask, int32_t key) {
    uint32_t s = hmix(key) & mask;
    while (true) {
        int32_t k = __ldcg(keys + s);
        if (k == key) return __ldcg(vals + s);
        if (k == -1) return 0;
        s = (s + 1) & mask;
    }
}

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

template <bool BIG>
__device__ __forceinline__ typename GainT<BIG>::T plm_gain(int64_t twoW, int64_t wD, int64_t wC, int64_t vu,
                                                           int64_t volD, int64_t volC) {
    using T = typename GainT<BIG>::T;
    return (T)twoW * (T)(wD - wC) - (T)vu * (T)(volD - volC + vu);
}

template <bool BIG>
using ValT = std::conditional_t<BIG, unsigned long long, unsigned int>;

// Warp-wide sums of per-lane counters, one atomic per warp.
__device__ __forceinline__ void add_counters(Counters *c, unsigned wanted, unsigned moved, unsigned entries,
                                             unsigned cand, unsigned dec) {
    wanted = __reduce_add_sync(0xffffffffu, wanted);
    moved = __reduce_add_sync(0xffffffffu, moved);
    entries = __reduce_add_sync(0xffffffffu, entries);
    cand = __reduce_add_sync(0xffffffffu, cand);
    dec = __reduce_add_sync(0xffffffffu, dec);
    if ((threadIdx.x & 31) == 0) {
        if (wanted) atomicAdd(&c->wanted, (unsigned long long)wanted);
        if (moved) atomicAdd(&c->moved, (unsigned long long)moved);
        if (entries) atomicAdd(&c->entries, (unsigned long long)entries);
        if (cand) atomicAdd(&c->candidates, (unsigned long long)cand);
        if (dec) atomicAdd(&c->decisions, (unsigned long long)dec);
    }
}

// Late sweeps: record a wanted move for the class's sequential re-check.
__device__ __forceinline__ void put_candidate(const SweepCtx &c, unsigned long long pos, int32_t u, int32_t C,
                                              int32_t D, int64_t wD, int64_t wC) {
    c.cand_u[pos] = u;
    c.cand_c[pos] = C;
    c.cand_d[pos] = D;
    c.cand_wd[pos] = wD;
    c.cand_wc[pos] = wC;
}

// ---------------------------------------------------------------------------
// Group kernel: G lanes per vertex.
// ---------------------------------------------------------------------------
template <int G, int DMAX, int WK, bool BIG, bool PLP>
__global__ void __launch_bounds__(kBlock) k_decide_group(SweepCtx c, const int32_t *__restrict__ list,
                                                         int64_t count) {
    using VT = ValT<BIG>;
    constexpr int SLOTS = 2 * DMAX;
    constexpr int GPB = kBlock / G;
    __shared__ int32_t s_keys[GPB * SLOTS];
    __shared__ VT s_vals[GPB * SLOTS];
    const int grp = threadIdx.x / G, gl = threadIdx.x % G, lane = threadIdx.x & 31;
    // groups are aligned runs of G lanes, so xor offsets below G stay inside
    // the group; the whole warp is converged at every shuffle
    const unsigned gmask = 0xffffffffu;
    int32_t *keys = s_keys + grp * SLOTS;
    VT *vals = s_vals + grp * SLOTS;

    const int64_t idx = (int64_t)blockIdx.x * GPB + grp;
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
    if (valid) {
        beg = c.g.rp[u];
        deg = (int)(c.g.rp[u + 1] - beg);
    }
#pragma unroll
    for (int k = gl; k < DMAX; k += G) {
        if (valid && k < deg) {
            const int32_t v = c.g.col[beg + k];
            const VT w = (VT)edge_weight<WK>(c.g.w, beg + k);
            tab_insert<VT>(keys, vals, SLOTS - 1, c.zeta[v], w);
        }
    }
    __syncwarp();
    const int32_t C = valid ? c.zeta[u] : 0;
    const int64_t wC = valid ? (int64_t)tab_lookup<VT>(keys, vals, SLOTS - 1, C) : 0;
    unsigned ncand = 0;
    if constexpr (!PLP) {
        const int64_t vu = valid ? c.g.vol[u] : 0;
        const int64_t volC = valid ? c.volc[C] : 0;
        const int64_t twoW = 2 * c.g.W;
        PlmBest<BIG> b;
        b.init();
#pragma unroll
        for (int s = gl; s < SLOTS; s += G) {
            const int32_t key = keys[s];
            if (valid && key >= 0) {
                ncand++;
                if (key != C)
                    b.offer(plm_gain<BIG>(twoW, (int64_t)vals[s], wC, vu, c.volc[key], volC), key, (int64_t)vals[s]);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) b.merge(b.shfl_xor(gmask, o));
        const bool want = gl == 0 && valid && b.id >= 0 && b.g > 0;
        const bool apply = want && !c.late;
        const unsigned ballot = __ballot_sync(0xffffffffu, want);
        unsigned long long base = 0;
        if (lane == 0 && ballot) base = atomicAdd(c.late ? c.ncand : c.nmv, (unsigned long long)__popc(ballot));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (want) {
            const unsigned long long pos = base + __popc(ballot & ((1u << lane) - 1u));
            if (apply) {
                c.zeta[u] = b.id;
                c.mv_u[pos] = u;
                c.mv_c[pos] = C;
            } else {
                put_candidate(c, pos, u, C, b.id, b.w, wC);
            }
        }
        add_counters(c.cnt, want, apply, gl == 0 && valid ? deg : 0, ncand, gl == 0 && valid);
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
        add_counters(c.cnt, 0, gl == 0 && adopt, gl == 0 && valid ? deg : 0, ncand, gl == 0 && valid);
    }
}

// ---------------------------------------------------------------------------
// Block kernel: one block per vertex (deg <= 1024).
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

template <int WK, bool BIG, bool PLP>
__global__ void __launch_bounds__(kBlock) k_decide_block(SweepCtx c, const int32_t *__restrict__ list,
                                                         int64_t count) {
    using VT = ValT<BIG>;
    __shared__ int32_t keys[BLK_SLOTS];
    __shared__ VT vals[BLK_SLOTS];
    __shared__ unsigned s_cand;
    using BT = std::conditional_t<PLP, PlpBest, PlmBest<BIG>>;
    __shared__ BT s_best[kBlock / 32];
    for (int64_t idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int32_t u = list[idx];
        bool valid = true;
        if constexpr (PLP) valid = c.active[u] != 0;
        if (!valid) continue;   // uniform across the block
        const int64_t beg = c.g.rp[u];
        const int deg = (int)(c.g.rp[u + 1] - beg);
        int slots = 64;
        while (slots < 2 * deg) slots <<= 1;
        const uint32_t mask = slots - 1;
        for (int s = threadIdx.x; s < slots; s += kBlock) { keys[s] = -1; vals[s] = 0; }
        if (threadIdx.x == 0) s_cand = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < deg; k += kBlock) {
            const int32_t v = c.g.col[beg + k];
            tab_insert<VT>(keys, vals, mask, c.zeta[v], (VT)edge_weight<WK>(c.g.w, beg + k));
        }
        __syncthreads();
        const int32_t C = c.zeta[u];
        const int64_t wC = (int64_t)tab_lookup<VT>(keys, vals, mask, C);
        unsigned ncand = 0;
        if constexpr (!PLP) {
            const int64_t vu = c.g.vol[u], volC = c.volc[C], twoW = 2 * c.g.W;
            PlmBest<BIG> b;
            b.init();
            for (int s = threadIdx.x; s < slots; s += kBlock) {
                const int32_t key = keys[s];
                if (key >= 0) {
                    ncand++;
                    if (key != C)
                        b.offer(plm_gain<BIG>(twoW, (int64_t)vals[s], wC, vu, c.volc[key], volC), key,
                                (int64_t)vals[s]);
                }
            }
            ncand = __reduce_add_sync(0xffffffffu, ncand);
            if ((threadIdx.x & 31) == 0) atomicAdd(&s_cand, ncand);
            b = block_best(b, s_best);
            if (threadIdx.x == 0) {
                const bool want = b.id >= 0 && b.g > 0;
                const bool apply = want && !c.late;
                if (apply) {
                    const unsigned long long pos = atomicAdd(c.nmv, 1ull);
                    c.zeta[u] = b.id;
                    c.mv_u[pos] = u;
                    c.mv_c[pos] = C;
                } else if (want) {
                    put_candidate(c, atomicAdd(c.ncand, 1ull), u, C, b.id, b.w, wC);
                }
                atomicAdd(&c.cnt->wanted, (unsigned long long)want);
                atomicAdd(&c.cnt->moved, (unsigned long long)apply);
                atomicAdd(&c.cnt->entries, (unsigned long long)deg);
                atomicAdd(&c.cnt->candidates, (unsigned long long)s_cand);
                atomicAdd(&c.cnt->decisions, 1ull);
            }
        } else {
            PlpBest b;
            b.init();
            for (int s = threadIdx.x; s < slots; s += kBlock) {
                const int32_t key = keys[s];
                if (key >= 0) {
                    ncand++;
                    b.offer((int64_t)vals[s], fmix32((uint32_t)key ^ c.tie_salt), key);
                }
            }
            ncand = __reduce_add_sync(0xffffffffu, ncand);
            if ((threadIdx.x & 31) == 0) atomicAdd(&s_cand, ncand);
            b = block_best(b, s_best);
            const bool adopt = b.id >= 0 && b.w > wC;
            if (adopt)
                for (int k = threadIdx.x; k < deg; k += kBlock) c.active[c.g.col[beg + k]] = 1;
            if (threadIdx.x == 0) {
                if (adopt) c.zeta[u] = b.id;
                else c.active[u] = 0;
                atomicAdd(&c.cnt->moved, (unsigned long long)adopt);
                atomicAdd(&c.cnt->entries, (unsigned long long)deg);
                atomicAdd(&c.cnt->candidates, (unsigned long long)s_cand);
                atomicAdd(&c.cnt->decisions, 1ull);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Hub kernels (deg > 1024).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_hub(const int32_t *prefix, int nhubs, int32_t b) {
    int lo = 0, hi = nhubs - 1;
    while (lo < hi) {            // last h with prefix[h] <= b
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int WK, bool BIG, bool PLP>
__global__ void __launch_bounds__(kBlock) k_hub_aggregate(SweepCtx c) {
    using VT = ValT<BIG>;
    __shared__ int32_t keys[BLK_SLOTS];
    __shared__ VT vals[BLK_SLOTS];
    __shared__ int s_last;
    const int h = find_hub(c.hub_b1, c.nhubs, blockIdx.x);
    const HubInfo hi = c.hubs[h];
    const int32_t u = hi.v;
    if constexpr (PLP) {
        if (!c.active[u]) return;   // whole block; H2 sees it too
    }
    const int j = blockIdx.x - c.hub_b1[h];
    const int64_t rb = c.g.rp[u], re = c.g.rp[u + 1];
    const int64_t beg = rb + (int64_t)j * HUB_CHUNK;
    const int64_t end = min(re, beg + HUB_CHUNK);
    for (int s = threadIdx.x; s < BLK_SLOTS; s += kBlock) { keys[s] = -1; vals[s] = 0; }
    __syncthreads();
    for (int64_t e = beg + threadIdx.x; e < end; e += kBlock)
        tab_insert<VT>(keys, vals, BLK_SLOTS - 1, c.zeta[c.g.col[e]], (VT)edge_weight<WK>(c.g.w, e));
    __syncthreads();
    int32_t *gk = c.hub_keys + hi.tab;
    VT *gv = static_cast<VT *>(c.hub_vals) + hi.tab;
    const uint32_t gmask = (uint32_t)(hi.slots - 1);
    for (int s = threadIdx.x; s < BLK_SLOTS; s += kBlock)
        if (keys[s] >= 0) tab_insert<VT>(gk, gv, gmask, keys[s], vals[s]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned done = atomicAdd(&c.hub_done1[h], 1u);
        s_last = (done == (unsigned)hi.nb1 - 1);
        atomicAdd(&c.cnt->entries, (unsigned long long)(end - beg));
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        c.hub_done1[h] = 0;
        static_cast<VT *>(c.hub_wc)[h] = tab_lookup_cg<VT>(gk, gv, gmask, c.zeta[u]);
    }
}

template <int WK, bool BIG, bool PLP>
__global__ void __launch_bounds__(kBlock) k_hub_decide(SweepCtx c) {
    using VT = ValT<BIG>;
    using BT = std::conditional_t<PLP, PlpBest, PlmBest<BIG>>;
    __shared__ BT s_best[kBlock / 32];
    __shared__ unsigned s_cand;
    __shared__ int s_last;
    const int h = find_hub(c.hub_b2, c.nhubs, blockIdx.x);
    const HubInfo hi = c.hubs[h];
    const int32_t u = hi.v;
    if constexpr (PLP) {
        if (!c.active[u]) return;
    }
    const int j = blockIdx.x - c.hub_b2[h];
    int32_t *gk = c.hub_keys + hi.tab;
    VT *gv = static_cast<VT *>(c.hub_vals) + hi.tab;
    const int64_t s0 = (int64_t)j * HUB_SCAN, s1 = min(hi.slots, s0 + HUB_SCAN);
    const int32_t C = c.zeta[u];
    const int64_t wC = (int64_t)static_cast<const VT *>(c.hub_wc)[h];
    if (threadIdx.x == 0) s_cand = 0;
    __syncthreads();
    unsigned ncand = 0;
    BT b;
    b.init();
    if constexpr (!PLP) {
        const int64_t vu = c.g.vol[u], volC = c.volc[C], twoW = 2 * c.g.W;
        for (int64_t s = s0 + threadIdx.x; s < s1; s += kBlock) {
            const int32_t key = gk[s];
            if (key >= 0) {
                ncand++;
                if (key != C) b.offer(plm_gain<BIG>(twoW, (int64_t)gv[s], wC, vu, c.volc[key], volC), key, (int64_t)gv[s]);
                gk[s] = -1;
                gv[s] = 0;
            }
        }
    } else {
        for (int64_t s = s0 + threadIdx.x; s < s1; s += kBlock) {
            const int32_t key = gk[s];
            if (key >= 0) {
                ncand++;
                b.offer((int64_t)gv[s], fmix32((uint32_t)key ^ c.tie_salt), key);
                gk[s] = -1;
                gv[s] = 0;
            }
        }
    }
    ncand = __reduce_add_sync(0xffffffffu, ncand);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_cand, ncand);
    b = block_best(b, s_best);
    const int64_t pslot = blockIdx.x;
    if (threadIdx.x == 0) {
        if constexpr (!PLP) {
            if constexpr (BIG) {
                c.part_g[pslot] = (int64_t)(uint64_t)b.g;
                c.part_g2[pslot] = (int64_t)(b.g >> 64);
            } else {
                c.part_g[pslot] = b.g;
            }
            c.part_w[pslot] = b.w;
        } else {
            c.part_g[pslot] = b.w;
            c.part_tk[pslot] = b.tk;
        }
        c.part_id[pslot] = b.id;
        atomicAdd(&c.cnt->candidates, (unsigned long long)s_cand);
        __threadfence();
        unsigned done = atomicAdd(&c.hub_done2[h], 1u);
        s_last = (done == (unsigned)hi.nb2 - 1);
    }
    __syncthreads();
    if (!s_last) return;
    if (threadIdx.x == 0) {
        __threadfence();
        c.hub_done2[h] = 0;
        BT r;
        r.init();
        const int64_t p0 = c.hub_b2[h];
        for (int k = 0; k < hi.nb2; k++) {
            BT o;
            o.id = __ldcg(c.part_id + p0 + k);
            if constexpr (!PLP) {
                if constexpr (BIG) {
                    uint64_t lo = (uint64_t)__ldcg(c.part_g + p0 + k);
                    uint64_t hi2 = (uint64_t)__ldcg(c.part_g2 + p0 + k);
                    o.g = (__int128)(((unsigned __int128)hi2 << 64) | lo);
                } else {
                    o.g = __ldcg(c.part_g + p0 + k);
                }
                o.w = __ldcg(c.part_w + p0 + k);
            } else {
                o.w = __ldcg(c.part_g + p0 + k);
                o.tk = __ldcg(c.part_tk + p0 + k);
            }
            r.merge(o);
        }
        const int deg = (int)(c.g.rp[u + 1] - c.g.rp[u]);
        if constexpr (!PLP) {
            const bool want = r.id >= 0 && r.g > 0;
            const bool apply = want && !c.late;
            if (apply) {
                const unsigned long long pos = atomicAdd(c.nmv, 1ull);
                c.zeta[u] = r.id;
                c.mv_u[pos] = u;
                c.mv_c[pos] = C;
            } else if (want) {
                put_candidate(c, atomicAdd(c.ncand, 1ull), u, C, r.id, r.w, wC);
            }
            atomicAdd(&c.cnt->wanted, (unsigned long long)want);
            atomicAdd(&c.cnt->moved, (unsigned long long)apply);
            s_best[0] = r;
        } else {
            bool adopt = r.id >= 0 && r.w > wC;
            if (adopt) c.zeta[u] = r.id;
            else c.active[u] = 0;
            atomicAdd(&c.cnt->moved, (unsigned long long)adopt);
            s_best[0] = r;
            s_last = adopt ? 2 : 1;
        }
        atomicAdd(&c.cnt->decisions, 1ull);
        (void)deg;
    }
    __syncthreads();
    if constexpr (PLP) {
        if (s_last == 2) {
            const int64_t rb = c.g.rp[u], re = c.g.rp[u + 1];
            for (int64_t e = rb + threadIdx.x; e < re; e += kBlock) c.active[c.g.col[e]] = 1;
        }
    }
}

// Applies the recorded moves of one class to the community volumes.
__global__ void k_apply_moves(const int32_t *mv_u, const int32_t *mv_c, const unsigned long long *nmv,
                              const int32_t *zeta, const int64_t *vol, int64_t *volc);

}  // namespace cd
