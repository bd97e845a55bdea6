// Persistent kernels: one cooperative launch runs whole PLM move phases
// (every sweep, every colour class) or whole PLP runs (every iteration) of
// one or many graphs.  A team of blocks works on one graph at a time: colour
// classes follow each other in order, one team barrier after each; inside a
// class, the team's blocks take the work items in serpentine passes (hub
// chunks, block items and lane groups first from the expensive end, then
// alternating), then the hub-decide slices.  The block
// that finishes the class last (a finish counter) writes the hubs' deferred
// labels in early PLM sweeps and runs the sequential re-check in late ones,
// before the class's barrier.
//
// The team barrier is a generation counter; a block that waits longer than
// BARRIER_TIMEOUT_NS sets an error flag and the team's blocks leave the
// kernel, which the host reports as CD_ETIMEOUT.
#pragma once
#include "barrier.cuh"
#include "move_kernels.cuh"

namespace cd {

constexpr int PHASE_SMEM = 32768;          // dynamic shared memory per block
static_assert(SMEM_BYTES <= PHASE_SMEM, "role tables exceed the phase kernels' shared memory");
constexpr int RC_SMALL = 4096;             // candidates sorted in shared memory
// Per-class schedule record (read by one thread per block at class start).
struct ClassMeta {
    int64_t off[NBINS + 1];    // bucket offsets into the schedule order
    int32_t h0, nhubs;         // first hub (global index), hubs of the class
    int32_t nb1, nb2;          // aggregation items, decide slices
    int32_t it0, sl0;          // first aggregation item / decide slice
    int32_t nrelax;            // hubs with more than HUB_RELAX neighbours
    int32_t pad;
};

struct PhaseArgs {
    GraphView g;
    int32_t *zeta;
    const int32_t *order;
    int32_t ncol;
    const int64_t *class_off;              // [ncol * NBINS + 1]
    const int32_t *class_hub0;             // [ncol + 1]
    const int32_t *class_nb1, *class_nb2;  // [ncol]
    const HubInfo *hubs;
    const int32_t *hb1, *hb2;
    const ChunkDesc *chunks;               // aggregation items, class by class
    const SliceDesc *slices;               // decide slices, class by class
    const ClassMeta *meta;                 // [ncol]
    int32_t *hub_occ;                      // occupied-slot lists, laid out like the hub tables
    unsigned int *hub_nocc;                // per hub
    int32_t *dz_u, *dz_l;                  // deferred hub label writes of the current class
    unsigned int *dz_n;                    //   and their count (0 between classes)
    int32_t *cstamp;                       // re-check: per community, last class step a hub moved it (0: never)
    int32_t *hub_keys;
    void *hub_vals, *hub_wc;
    unsigned int *done1, *done2;
    int64_t *part_g, *part_g2, *part_w;
    int32_t *part_id;
    uint32_t *part_tk;
    Counters *cnt;                         // one per sweep / iteration
    int32_t *result;                       // [0] sweeps / iterations run, [1] converged
    // PLM
    int64_t *vol_a, *vol_b;                // launch t reads vol[t & 1], writes vol[(t+1) & 1]
    int32_t *mv_u, *mv_c, *cd;
    int64_t *cwd, *cwc;
    unsigned long long *nmv;               // [2][ncol]
    unsigned long long *ncand;             // [ncol]
    uint64_t *tmp_a, *tmp_b;
    int32_t ubits;
    int32_t *rc_u;
    uint64_t *rc_cd, *rc_vu;
    int64_t *rc_dw;
    int32_t max_sweeps, recheck_from;
    int64_t res_p, res_q;                  // resolution gamma = res_p / res_q of the gain (1 / 1: modularity)
    int32_t racy;                          // racy schedule: live volumes (read and written in vol_a), no
    int32_t pad_racy;                      //   replay, no re-check
    // PLP
    uint8_t *active;
    unsigned long long *sched;             // [1] class finish counter (starts at 0)
    uint64_t seed;
    double theta;
    int32_t max_iters;
    // profile mode: block 0 adds the wall time of each class stage (ns):
    // [0] items (+ barrier), [1] hub decide (+ barrier), [2] re-check (+ barrier)
    unsigned long long *stage_ns;
    // class trace (profile level 2): block 0 stamps the global timer when the
    // phase starts ([0]) and after the barrier of class k in sweep sw
    // ([1 + sw * ncol + k]); skipped (empty) classes keep 0
    unsigned long long *class_ns;
    // with class_ns: STAGE_SLOTS words per class step (ST_* below): the latest
    // time any block finished its items, its hub-decide slices and the
    // finisher's work, and the longest single item of each kind
    unsigned long long *stage_max;
};

// SweepCtx of class k (layout, roles, hubs).
__device__ __forceinline__ int32_t class_ctx(const PhaseArgs &a, int32_t k, SweepCtx &c) {
    const ClassMeta m = a.meta[k];
    const int64_t base = m.off[0];
    c.order = a.order + base;
    for (int b = 0; b <= NBINS; b++) c.off[b] = m.off[b] - base;
    const int32_t h0 = m.h0;
    c.nhubs = m.nhubs;
    c.hubs = a.hubs + h0;
    c.hub_b1 = a.hb1 + h0;
    c.hub_b2 = a.hb2 + h0;
    c.chunks = a.chunks + m.it0;
    c.slices = a.slices + m.sl0;
    c.hub_occ = a.hub_occ;
    c.hub_nocc = a.hub_nocc + h0;
    c.hub_keys = a.hub_keys;
    c.hub_vals = a.hub_vals;
    c.hub_wc = static_cast<char *>(a.hub_wc) + (size_t)h0 * 8;
    c.hub_done1 = a.done1 + h0;
    c.hub_done2 = a.done2 + h0;
    c.part_g = a.part_g;
    c.part_g2 = a.part_g2;
    c.part_w = a.part_w;
    c.part_id = a.part_id;
    c.part_tk = a.part_tk;
    const int64_t n0 = c.off[1] - c.off[0], n1 = c.off[2] - c.off[1], n2 = c.off[3] - c.off[2];
    const int64_t n3 = c.off[4] - c.off[3], n4 = c.off[5] - c.off[4];
    c.bend[0] = (int32_t)((n0 + kBlock / 4 - 1) / (kBlock / 4));
    c.bend[1] = c.bend[0] + (int32_t)((n1 + kBlock / 8 - 1) / (kBlock / 8));
    c.bend[2] = c.bend[1] + (int32_t)((n2 + kBlock / 32 - 1) / (kBlock / 32));
    c.bend[3] = c.bend[2] + (int32_t)n3;
    c.bend[4] = c.bend[3] + (int32_t)n4;
    c.bend[5] = c.bend[4] + m.nb1;
    c.nrelax = m.nrelax;
    c.dz_u = a.dz_u;
    c.dz_l = a.dz_l;
    c.dz_n = a.dz_n;
    return m.nb2;
}

template <int WK, bool BIG, bool PLP>
__device__ __forceinline__ void run_item(const SweepCtx &c, int32_t b, unsigned char *smem,
                                         typename BestOf<PLP, BIG>::T *s_best, unsigned *s_cand, int *s_last) {
    if (b < c.bend[0]) role_group<4, 4, WK, BIG, PLP>(c, b, c.order + c.off[0], c.off[1] - c.off[0], smem);
    else if (b < c.bend[1]) role_group<8, 16, WK, BIG, PLP>(c, b - c.bend[0], c.order + c.off[1], c.off[2] - c.off[1], smem);
    else if (b < c.bend[2]) role_group<32, 128, WK, BIG, PLP>(c, b - c.bend[1], c.order + c.off[2], c.off[3] - c.off[2], smem);
    else if (b < c.bend[3]) role_block<WK, BIG, PLP, false>(c, b - c.bend[2], c.order + c.off[3], smem, s_best, s_cand);
    else if (b < c.bend[4]) role_block<WK, BIG, PLP, true>(c, b - c.bend[3], c.order + c.off[4], smem, s_best, s_cand);
    else role_hub_aggregate<WK, BIG, PLP>(c, b - c.bend[4], smem, s_best, s_last);
}

// Hub decide: slice `item` of a hub table; the last slice of a hub decides.
// A PLM slice ranks the candidates D != C by 2W q omega(u,D) - p vol(u) vol(D)
// (gamma = p / q), which differs from the gain only by a term that is the
// same for every D,
// so the slices need not know omega(u, C); the slice that finds C in the
// table records omega(u, C) for the last slice, which completes the gain of
// the best candidate.  The hub's aggregation is complete when the slice
// runs (wait_hub_ready).
template <int WK, bool BIG, bool PLP>
__device__ __forceinline__ void role_hub_decide(const SweepCtx &c, int32_t item, typename BestOf<PLP, BIG>::T *s_best,
                                                unsigned *s_cand, int *s_last) {
    using VT = ValT<BIG>;
    using BT = typename BestOf<PLP, BIG>::T;
    const SliceDesc hi = c.slices[item];
    const int h = hi.h;
    const int32_t u = hi.u;
    if constexpr (PLP) {
        if (!hi.relax && !c.racy && !c.active[u]) return;
    }
    const HubTable<VT> tb(c.hub_keys, c.hub_vals, hi.tab);
    const int32_t *occ = c.hub_occ + hi.tab;
    const int64_t nocc = (int64_t)__ldcg(c.hub_nocc + h);
    const int64_t s0 = hi.s0, s1 = min(hi.s1, nocc);
    const int32_t C = c.zeta[u];
    VT *hwc = static_cast<VT *>(c.hub_wc) + h;
    if (threadIdx.x == 0) *s_cand = 0;
    __syncthreads();
    unsigned ncand = 0;
    BT b;
    b.init();
    int64_t vu = 0;
    if constexpr (!PLP) vu = c.g.vol[u];
    const int64_t twoW = 2 * c.g.W;
    // four occupied slots per thread and step: slot numbers, then the slots,
    // then candidate volumes, then gains (every slot of the list is read and
    // emptied by one thread of one slice)
    for (int64_t i0 = s0 + threadIdx.x; i0 < s1; i0 += 4 * kBlock) {
        int32_t sl[4], ky[4];
        int64_t wv[4], vk[4];
#pragma unroll
        for (int j = 0; j < 4; j++) sl[j] = i0 + j * kBlock < s1 ? __ldcg(occ + i0 + j * kBlock) : -1;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            ky[j] = -1;
            wv[j] = 0;
            if (sl[j] >= 0) tb.read(sl[j], ky[j], wv[j]);
        }
        if constexpr (!PLP) {
            using T = typename GainT<BIG>::T;
#pragma unroll
            for (int j = 0; j < 4; j++) vk[j] = (sl[j] >= 0 && ky[j] != C) ? c.volc[ky[j]] : 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (sl[j] < 0) continue;
                ncand++;
                if (ky[j] != C) b.offer((T)twoW * (T)c.res_q * (T)wv[j] - (T)c.res_p * (T)vu * (T)vk[j], ky[j], wv[j]);
                else { *hwc = (VT)wv[j]; __threadfence(); }
                tb.clear(sl[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (sl[j] < 0) continue;
                ncand++;
                b.offer(wv[j], fmix32((uint32_t)ky[j] ^ c.tie_salt), ky[j]);
                if (ky[j] == C) { *hwc = (VT)wv[j]; __threadfence(); }
                tb.clear(sl[j]);
            }
        }
    }
    ncand = __reduce_add_sync(0xffffffffu, ncand);
    if ((threadIdx.x & 31) == 0) atomicAdd(s_cand, ncand);
    b = block_best(b, s_best);
    if (threadIdx.x == 0) {
        if constexpr (!PLP) {
            if constexpr (BIG) {
                c.part_g[item] = (int64_t)(uint64_t)b.g;
                c.part_g2[item] = (int64_t)(b.g >> 64);
            } else {
                c.part_g[item] = b.g;
            }
            c.part_w[item] = b.w;
        } else {
            c.part_g[item] = b.w;
            c.part_tk[item] = b.tk;
        }
        c.part_id[item] = b.id;
        c.bcnt[BC_CAND] += *s_cand;
        __threadfence();
        const unsigned done = atomicAdd(&c.hub_done2[h], 1u);
        *s_last = (done == (unsigned)hi.nb2 - 1);
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    {   // merge the partial bests of every slice of this hub
        BT r;
        r.init();
        const int64_t p0 = hi.p0;
        for (int k = threadIdx.x; k < hi.nb2; k += kBlock) {
            BT o;
            o.id = __ldcg(c.part_id + p0 + k);
            if constexpr (!PLP) {
                if constexpr (BIG) {
                    const uint64_t lo = (uint64_t)__ldcg(c.part_g + p0 + k);
                    const uint64_t hi2 = (uint64_t)__ldcg(c.part_g2 + p0 + k);
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
        b = block_best(r, s_best);
    }
    // omega(u, C) is 0 when no neighbour is in C (no slice recorded it)
    const int64_t wC = (int64_t)__ldcg(hwc);
    if constexpr (!PLP) {
        using T = typename GainT<BIG>::T;
        if (b.id >= 0)
            b.g = b.g - (T)(2 * c.g.W) * (T)c.res_q * (T)wC + (T)c.res_p * (T)c.g.vol[u] * (T)(c.volc[C] - c.g.vol[u]);
    }
    __syncthreads();   // every thread has read omega(u, C)
    if (threadIdx.x == 0) {
        c.hub_done2[h] = 0;
        c.hub_done1[h] = 0;
        c.hub_nocc[h] = 0;
        *hwc = 0;
    }
    hub_finish<BIG, PLP>(c, u, C, wC, b, s_last, hi.relax != 0);
}

// Spins (thread 0, bounded by BARRIER_TIMEOUT_NS) until every aggregation
// item of the hub of decide slice `item` has merged its chunk.  The caller
// has finished all of its own items, and items never wait, so the wait
// ends.  Returns false on a timeout (or a failure elsewhere in the team).
template <bool PLP>
__device__ __forceinline__ bool wait_hub_ready(const SweepCtx &c, int32_t item, GridBarrier *bar, int *s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const SliceDesc d = c.slices[item];
        const int h = d.h;
        const int32_t u = d.u;
        const unsigned need = (unsigned)d.nb1;
        bool skip = false;
        if constexpr (PLP) skip = !d.relax && !c.racy && !c.active[u];   // inactive hubs are neither aggregated nor decided
        if (!skip) {
            const uint64_t t0 = global_ns();
            while (__ldcg(c.hub_done1 + h) != need) {
                if (*(volatile int *)&bar->err != 0) { ok = 0; break; }
                if (global_ns() - t0 > BARRIER_TIMEOUT_NS) { atomicExch(&bar->err, 1); ok = 0; break; }
                __nanosleep(64);
            }
            __threadfence();
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Sequential re-check of one class's wanted moves, by one block.  The
// candidates are sorted by vertex id (one warp's shuffle network up to 32,
// a bitonic network in shared memory up to RC_SMALL, else a block-wide LSD
// radix sort in global scratch), and the whole block gathers their records
// in that order.  Warp 0 then walks them in windows of 32, accepting in each
// round the lowest lane whose gain, on the volumes as updated by every move
// accepted before it, is positive; the later lanes of the window adjust
// their copies of the volumes they share with an accepted move.  Accepted
// moves update zeta and the volumes before the next window loads its
// volumes; the records themselves never change and are read a window ahead.
// ---------------------------------------------------------------------------
struct RecheckArgs {
    const int32_t *cu, *cc, *cd;
    const int64_t *cwd, *cwc;
    const unsigned long long *ncand;
    int32_t *zeta;
    const int64_t *vol;
    int64_t *volc;
    int64_t twoW;
    int64_t res_p, res_q;      // resolution gamma = res_p / res_q
    uint64_t *tmp_a, *tmp_b;   // class-sized scratch for long candidate lists
    int ubits;                 // bits of the largest vertex id
    int32_t *rc_u;             // class-sized: the candidates' records in id order
    uint64_t *rc_cd, *rc_vu;   //   (C | D << 32), vol(u) | hub << 63
    int64_t *rc_dw;            //   omega(u, D) - omega(u, C)
    Counters *cnt;
    const int64_t *rp;         // row offsets (hub test)
    int32_t *cstamp;           // cstamp[X] == step: a hub of this class moved into or out of X
    int32_t step;              // id of this class step (> 0)
    unsigned long long *stage_ns;   // profile mode: [1] += sort time; else nullptr
    // racy schedule: candidates of a round may be adjacent.  Every accepted
    // mover stamps its neighbours (cstamp is then indexed by vertex), and a
    // candidate stamped earlier in the round waits for the next sweep: only a
    // moving neighbour changes omega(u, C) or omega(u, D), so the gains of
    // the candidates that go ahead are exact.
    int32_t nbr_stamp;
    const int32_t *col;        // adjacency (neighbour stamps)
};


__device__ __forceinline__ void rc_radix_pass(const uint64_t *in, uint64_t *out, int64_t m, int shift,
                                              unsigned char *smem) {
    constexpr int NW = kBlock / 32;
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(smem);                          // [NW][256]
    int64_t *base = reinterpret_cast<int64_t *>(smem + NW * 256 * 4);            // [256]
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + NW * 256 * 4 + 256 * 8);  // [256]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 256) hist[tid] = 0;
    for (int j = tid; j < NW * 256; j += kBlock) wcnt[j] = 0;
    __syncthreads();
#pragma unroll 4
    for (int64_t i = tid; i < m; i += kBlock) atomicAdd(&hist[(uint32_t)(in[i] >> shift) & 255u], 1u);
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int d = 0; d < 256; d++) { base[d] = run; run += hist[d]; }
    }
    __syncthreads();
    // the next round's key is loaded before this round's barriers
    uint64_t knext = tid < m ? in[tid] : 0;
    for (int64_t r = 0; r < m; r += kBlock) {
        const int64_t i = r + tid;
        const bool valid = i < m;
        const uint64_t k = knext;
        if (i + kBlock < m) knext = in[i + kBlock];
        const uint32_t d = valid ? ((uint32_t)(k >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp * 256 + d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int j = 0; j < NW; j++) {
            const uint32_t cc = wcnt[j * 256 + tid];
            wcnt[j * 256 + tid] = run;
            run += cc;
        }
        __syncthreads();
        if (valid) out[base[d] + wcnt[warp * 256 + d] + rank] = k;
        __syncthreads();
        base[tid] += run;
        for (int j = 0; j < NW; j++) wcnt[j * 256 + tid] = 0;
        __syncthreads();
    }
}

// One re-check candidate as warp 0 walks it: its record, and the volumes of
// its two communities and its hub block flag as of the start of its window.
struct RcLane {
    int32_t C, D, u;
    int64_t vu, dw;
    bool hub;
};

__device__ __forceinline__ RcLane rc_load(const RecheckArgs &a, int64_t i, int64_t m) {
    RcLane r{-1, -2, 0, 0, 0, false};
    if (i < m) {
        const uint64_t cd = __ldcg(a.rc_cd + i), vh = __ldcg(a.rc_vu + i);
        r.C = (int32_t)(uint32_t)cd;
        r.D = (int32_t)(cd >> 32);
        r.vu = (int64_t)(vh & ~(1ull << 63));
        r.hub = (vh >> 63) != 0;
        r.dw = __ldcg(a.rc_dw + i);
        r.u = __ldcg(a.rc_u + i);
    }
    return r;
}

// Walk of the sorted candidates by warp 0 (deterministic schedule), in
// windows of 32 as described above, with the volume and stamp reads taken
// off the sequential path: the reads for window w + 1 are issued when window
// w starts (they see every move of the windows before w, which are committed
// by then), and each move that window w accepts is folded into them as a
// volume difference (and, for hubs, as the stamp it would have written), so
// that window w + 1 starts from exactly the state the sequential order gives
// it.  Records are read two windows ahead.
template <bool BIG>
__device__ __forceinline__ void recheck_walk_pipelined(const RecheckArgs &a, int64_t m) {
    const int lane = threadIdx.x & 31;
    unsigned long long moved = 0;
    RcLane cur = rc_load(a, lane, m), nxt = rc_load(a, 32 + lane, m);
    int64_t volC = cur.C >= 0 ? __ldcg(a.volc + cur.C) : 0, volD = cur.C >= 0 ? __ldcg(a.volc + cur.D) : 0;
    bool blocked = cur.hub && (__ldcg(a.cstamp + cur.C) == a.step || __ldcg(a.cstamp + cur.D) == a.step);
    for (int64_t w0 = 0; w0 < m; w0 += 32) {
        const bool valid = w0 + lane < m;
        // next window: its volumes and stamps as of now, then the records after it
        const bool nvalid = nxt.C >= 0;
        const int64_t nvC = nvalid ? __ldcg(a.volc + nxt.C) : 0, nvD = nvalid ? __ldcg(a.volc + nxt.D) : 0;
        const bool nstamped =
            nxt.hub && (__ldcg(a.cstamp + nxt.C) == a.step || __ldcg(a.cstamp + nxt.D) == a.step);
        const RcLane nn = rc_load(a, w0 + 64 + lane, m);
        int64_t dC = 0, dD = 0;
        bool nblk = false;
        bool mine = false;
        unsigned pending = __ballot_sync(0xffffffffu, valid);
        while (pending) {
            const bool acc = ((pending >> lane) & 1u) && !blocked &&
                             plm_gain<BIG>(a.twoW, a.res_q, a.res_p, cur.dw, 0, cur.vu, volD, volC) > 0;
            const unsigned am = __ballot_sync(0xffffffffu, acc);
            if (am == 0) break;
            const int k = __ffs(am) - 1;
            pending &= ~(0xffffffffu >> (31 - k));   // lanes 0..k are decided
            const int32_t Ck = __shfl_sync(0xffffffffu, cur.C, k), Dk = __shfl_sync(0xffffffffu, cur.D, k);
            const int64_t vk = __shfl_sync(0xffffffffu, cur.vu, k);
            const bool hk = __shfl_sync(0xffffffffu, (int)cur.hub, k) != 0;
            if (lane == k) {
                mine = true;
                if (cur.hub) {
                    a.cstamp[cur.C] = a.step;
                    a.cstamp[cur.D] = a.step;
                }
            } else if (lane > k) {
                if (cur.C == Ck) volC -= vk; else if (cur.C == Dk) volC += vk;
                if (cur.D == Ck) volD -= vk; else if (cur.D == Dk) volD += vk;
                if (hk && cur.hub && (cur.C == Ck || cur.C == Dk || cur.D == Ck || cur.D == Dk)) blocked = true;
            }
            // every candidate of the next window comes after this move
            if (nxt.C == Ck) dC -= vk; else if (nxt.C == Dk) dC += vk;
            if (nxt.D == Ck) dD -= vk; else if (nxt.D == Dk) dD += vk;
            if (hk && nxt.hub && (nxt.C == Ck || nxt.C == Dk || nxt.D == Ck || nxt.D == Dk)) nblk = true;
        }
        // the next window's volume reads are ordered before this window's
        // commits (a stamp written above may or may not be seen by them:
        // nblk holds it either way)
        __syncwarp();
        if (valid && mine) {
            a.zeta[cur.u] = cur.D;
            vol_add(a.volc, cur.C, -cur.vu);
            vol_add(a.volc, cur.D, cur.vu);
        }
        moved += __popc(__ballot_sync(0xffffffffu, valid && mine));
        __syncwarp();
        cur = nxt;
        volC = nvC + dC;
        volD = nvD + dD;
        blocked = nstamped || nblk;
        nxt = nn;
    }
    if (lane == 0 && moved) atomicAdd(&a.cnt->moved, moved);
}

template <bool BIG>
__device__ __noinline__ void recheck_block(const RecheckArgs &a, unsigned char *smem) {
    const int64_t m = (int64_t)__ldcg(a.ncand);
    if (m == 0) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t t_sort = a.stage_ns && tid == 0 ? global_ns() : 0;
    const uint64_t *keys;
    if (m <= 32) {
        // one warp: bitonic network over the lanes, no block barriers
        uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
        if (tid < 32) {
            uint64_t x = lane < m ? (((uint64_t)(uint32_t)__ldcg(a.cu + lane) << 32) | (uint32_t)lane) : ~0ull;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, x, j);
                    const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                    x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
                }
            sk[lane] = x;
        }
        __syncthreads();
        keys = sk;
    } else if (m <= RC_SMALL) {
        uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
        int P = 1;
        while (P < m) P <<= 1;
        for (int i = tid; i < P; i += kBlock)
            sk[i] = i < m ? (((uint64_t)(uint32_t)__ldcg(a.cu + i) << 32) | (uint32_t)i) : ~0ull;
        __syncthreads();
        // bitonic network: stages whose partner is in the same warp (j < 32)
        // run on registers with shuffles, the others through shared memory
        const int wbase = tid & ~31;
        auto warp_stages = [&](int k_lo, int k_hi, int j_top) {
            for (int i0 = wbase; i0 < P; i0 += kBlock) {   // whole warps: P is a multiple of 64
                const int i = i0 + lane;
                uint64_t x = sk[i];
                for (int k = k_lo; k <= k_hi; k <<= 1)
                    for (int j = min(k >> 1, j_top); j > 0; j >>= 1) {
                        const uint64_t y = __shfl_xor_sync(0xffffffffu, x, j);
                        const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
                        x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
                    }
                sk[i] = x;
            }
            __syncthreads();
        };
        warp_stages(2, 32, 16);
        for (int k = 64; k <= P; k <<= 1) {
            for (int j = k >> 1; j >= 32; j >>= 1) {
                for (int i = tid; i < P; i += kBlock) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const bool up = (i & k) == 0;
                        const uint64_t x = sk[i], y = sk[ixj];
                        if ((x > y) == up) { sk[i] = y; sk[ixj] = x; }
                    }
                }
                __syncthreads();
            }
            warp_stages(k, k, 16);
        }
        keys = sk;
    } else {
        for (int64_t i = tid; i < m; i += kBlock)
            a.tmp_a[i] = ((uint64_t)(uint32_t)__ldcg(a.cu + i) << 32) | (uint32_t)i;
        __syncthreads();
        uint64_t *src = a.tmp_a, *dst = a.tmp_b;
        for (int shift = 32; shift < 32 + a.ubits; shift += 8) {
            rc_radix_pass(src, dst, m, shift, smem);
            uint64_t *t = src;
            src = dst;
            dst = t;
        }
        __syncthreads();
        keys = src;
    }
    if (a.stage_ns && tid == 0) atomicAdd(a.stage_ns + 1, global_ns() - t_sort);
    // the whole block gathers the candidates' records in id order, so that
    // the walk below reads them contiguously
#pragma unroll 4
    for (int64_t i = tid; i < m; i += kBlock) {
        const uint32_t ci = (uint32_t)(keys[i] & 0xffffffffull);
        const int32_t u = __ldcg(a.cu + ci);
        const uint32_t C = (uint32_t)__ldcg(a.cc + ci), D = (uint32_t)__ldcg(a.cd + ci);
        const bool hub = !a.nbr_stamp && a.rp[u + 1] - a.rp[u] > HUB_RELAX;
        a.rc_u[i] = u;
        a.rc_cd[i] = ((uint64_t)D << 32) | C;
        a.rc_vu[i] = (uint64_t)a.vol[u] | ((uint64_t)hub << 63);
        a.rc_dw[i] = __ldcg(a.cwd + ci) - __ldcg(a.cwc + ci);
    }
    __syncthreads();
    if (tid < 32 && !a.nbr_stamp) {
        recheck_walk_pipelined<BIG>(a, m);
    } else if (tid < 32) {
        unsigned long long moved = 0;
        // records are read one window ahead; they never change, only the
        // volumes and stamps do, and those are read after the previous
        // window's moves are committed
        uint64_t n_cd = lane < m ? __ldcg(a.rc_cd + lane) : 0, n_vu = lane < m ? __ldcg(a.rc_vu + lane) : 0;
        int64_t n_dw = lane < m ? __ldcg(a.rc_dw + lane) : 0;
        int32_t n_u = lane < m ? __ldcg(a.rc_u + lane) : 0;
        for (int64_t w0 = 0; w0 < m; w0 += 32) {
            const bool valid = w0 + lane < m;
            const int32_t C = valid ? (int32_t)(uint32_t)n_cd : -1, D = valid ? (int32_t)(n_cd >> 32) : -2;
            const int64_t vu = (int64_t)(n_vu & ~(1ull << 63)), dw = n_dw;
            const bool hub = valid && (n_vu >> 63);
            const int32_t u = n_u;
            const int64_t j = w0 + 32 + lane;
            if (j < m) {
                n_cd = __ldcg(a.rc_cd + j);
                n_vu = __ldcg(a.rc_vu + j);
                n_dw = __ldcg(a.rc_dw + j);
                n_u = __ldcg(a.rc_u + j);
            }
            int64_t volC = valid ? __ldcg(a.volc + C) : 0;
            int64_t volD = valid ? __ldcg(a.volc + D) : 0;
            // a hub whose omega(u, C) or omega(u, D) a hub moved earlier in
            // this class may have changed waits for the next sweep
            bool blocked = hub && (__ldcg(a.cstamp + C) == a.step || __ldcg(a.cstamp + D) == a.step);
            if (a.nbr_stamp) blocked = valid && __ldcg(a.cstamp + u) == a.step;
            bool mine = false;
            // Every undecided lane evaluates its gain with the volumes as
            // updated by the moves accepted so far.  The lowest accepting lane
            // is accepted: every lane below it was evaluated on exactly the
            // state the sequential order gives it and declined, so it is done
            // too.  Lanes above it fold the accepted move into their volumes
            // and evaluate again.  A window thus costs one round per accepted
            // move (plus one), not one per candidate.
            unsigned pending = __ballot_sync(0xffffffffu, valid);
            while (pending) {
                const bool acc = ((pending >> lane) & 1u) && !blocked &&
                                 plm_gain<BIG>(a.twoW, a.res_q, a.res_p, dw, 0, vu, volD, volC) > 0;
                const unsigned am = __ballot_sync(0xffffffffu, acc);
                if (am == 0) break;
                const int k = __ffs(am) - 1;
                pending &= ~(0xffffffffu >> (31 - k));   // lanes 0..k are decided
                const int32_t Ck = __shfl_sync(0xffffffffu, C, k), Dk = __shfl_sync(0xffffffffu, D, k);
                const int64_t vk = __shfl_sync(0xffffffffu, vu, k);
                const bool hk = __shfl_sync(0xffffffffu, (int)hub, k) != 0;
                if (lane == k) {
                    mine = true;
                    if (hub) {
                        a.cstamp[C] = a.step;
                        a.cstamp[D] = a.step;
                    }
                } else if (lane > k) {
                    if (C == Ck) volC -= vk; else if (C == Dk) volC += vk;
                    if (D == Ck) volD -= vk; else if (D == Dk) volD += vk;
                    if (hk && hub && (C == Ck || C == Dk || D == Ck || D == Dk)) blocked = true;
                }
                if (a.nbr_stamp) {
                    // the whole warp stamps the accepted mover's neighbours
                    const int32_t uk = __shfl_sync(0xffffffffu, u, k);
                    const int64_t e1 = a.rp[uk + 1];
                    for (int64_t e = a.rp[uk] + lane; e < e1; e += 32) a.cstamp[a.col[e]] = a.step;
                    __syncwarp();
                    if (lane > k && !blocked) blocked = __ldcg(a.cstamp + u) == a.step;
                }
            }
            if (valid && mine) {
                a.zeta[u] = D;
                vol_add(a.volc, C, -vu);
                vol_add(a.volc, D, vu);
            }
            moved += __popc(__ballot_sync(0xffffffffu, valid && mine));
            __syncwarp();
        }
        if (lane == 0 && moved) atomicAdd(&a.cnt->moved, moved);
    }
    __syncthreads();
}

// PLP ties between dominant labels follow fmix32(label ^ salt), a seeded
// pseudo-random order that changes every iteration ("ties arbitrarily",
// Section III-A).
__device__ __forceinline__ uint32_t plp_salt_dev(uint64_t seed, int32_t it) {
    return fmix32(seed_word(seed) ^ (0x9E3779B9u * (uint32_t)(it + 1)));
}

// Per-block shared state of the phase bodies.
template <typename BT>
struct BlockShared {
    unsigned char *smem;       // dynamic PHASE_SMEM bytes
    BT *best;                  // [kBlock / 32]
    unsigned *cand, *gen;
    int *last, *ok, *nb2;
    long long *grab;           // decide slice taken by the block
    SweepCtx *c;
    unsigned long long *bcnt;  // [BC_N] the block's counter sums of the current sweep
};

// True in the block that finishes the class last (every block of the team
// calls it once per class; the counter only grows, fin_base tracks it).
__device__ __forceinline__ bool class_finisher(const PhaseArgs &a, const Team &tm, unsigned long long &fin_base,
                                               int *s_flag) {
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long f = atomicAdd(a.sched + 1, 1ull);
        *s_flag = f == fin_base + (unsigned long long)tm.size - 1;
    }
    __syncthreads();
    const bool last = *s_flag != 0;
    fin_base += (unsigned long long)tm.size;
    if (last) __threadfence();
    return last;
}

// Writes the labels that hubs of the class deferred (one block).
__device__ __forceinline__ void apply_deferred_labels(const SweepCtx &c) {
    const unsigned nd = __ldcg(c.dz_n);
    for (unsigned i = threadIdx.x; i < nd; i += kBlock) c.zeta[__ldcg(c.dz_u + i)] = __ldcg(c.dz_l + i);
    __syncthreads();
    if (threadIdx.x == 0 && nd) *c.dz_n = 0;
}

// Hub-decide slices of a class: block r of the team takes slices r, r +
// size, ... once it has finished its own items (so that no block waits for a
// hub chunk that it holds itself).
template <int WK, bool BIG, bool PLP, typename BT>
__device__ __forceinline__ bool decide_pool(const Team &tm, const SweepCtx &c, int32_t nb2,
                                            const BlockShared<BT> &sh, unsigned long long *smx = nullptr) {
    for (int32_t g = tm.rank; g < nb2; g += tm.size) {
        const uint64_t ti = smx && threadIdx.x == 0 ? global_ns() : 0;
        if (!wait_hub_ready<PLP>(c, g, tm.bar, sh.ok)) return false;
        const uint64_t tw = smx && threadIdx.x == 0 ? global_ns() : 0;
        role_hub_decide<WK, BIG, PLP>(c, g, sh.best, sh.cand, sh.last);
        if (smx && threadIdx.x == 0) {
            atomicMax(smx + ST_SLICE_WAIT, tw - ti);
            atomicMax(smx + ST_SLICE, global_ns() - tw);
        }
    }
    return true;
}

// Item of pass p for team block `rank` (-1: none).  The items of a class are
// ordered roughly by cost (lane groups, block items, hub chunks: the most
// expensive at the end), and the team walks them in a serpentine: pass 0
// hands the last `size` items out from the end, pass 1 the next `size` from
// their low end, and so on, so that a block that drew an expensive item in
// one pass draws a cheap one in the next.
__device__ __forceinline__ int32_t serpentine_item(int32_t p, int32_t rank, int32_t size, int32_t nit) {
    const int64_t hi = (int64_t)nit - (int64_t)p * size, lo = hi - size;
    const int64_t i = (p & 1) == 0 ? hi - 1 - rank : lo + rank;
    return i >= 0 && i < hi ? (int32_t)i : -1;
}

// ---------------------------------------------------------------------------
// PLM move phase (Algorithm 2) of one graph, run by one team: sweeps until
// no vertex wants to move.  Returns false when a barrier failed.
// ---------------------------------------------------------------------------
template <int WK, bool BIG>
__device__ bool move_phase_body(const PhaseArgs &a, const Team &tm, const BlockShared<PlmBest<BIG>> &sh,
                                int32_t *gt_keys, void *gt_vals) {
    SweepCtx &c = *sh.c;
    int64_t *vb[2] = {a.vol_a, a.vol_b};
    int64_t t = 0;
    int32_t prev_k = -1, prev_par = 0;
    int32_t sw = 0;
    int conv = 0;
    unsigned long long fin_base = 0;   // same in every block of the team
    const int64_t gtid = (int64_t)tm.rank * kBlock + threadIdx.x, gthreads = (int64_t)tm.size * kBlock;
    const bool tracer = a.class_ns && tm.rank == 0 && threadIdx.x == 0;
    if (tracer) a.class_ns[0] = global_ns();
    for (; sw < a.max_sweeps; sw++) {
        const int par = sw & 1;
        const int late = sw >= a.recheck_from;
        if (!late)
            for (int64_t i = gtid; i < a.ncol; i += gthreads) a.nmv[par * a.ncol + i] = 0;
        else
            for (int64_t i = gtid; i < a.ncol; i += gthreads) a.ncand[i] = 0;
        if (!team_sync(tm, sh.gen, sh.ok)) return false;
        for (int32_t k = 0; k < a.ncol; k++) {
            const int64_t cb = a.class_off[(int64_t)k * NBINS], ce = a.class_off[(int64_t)k * NBINS + NBINS];
            if (ce == cb) continue;
            __syncthreads();   // every thread is done with the previous class's context
            if (threadIdx.x == 0) {
                *sh.nb2 = class_ctx(a, k, c);
                c.g = a.g;
                c.zeta = a.zeta;
                c.gt_keys = gt_keys;
                c.gt_vals = gt_vals;
                c.cnt = a.cnt + sw;
                c.bcnt = sh.bcnt;
                c.res_p = a.res_p;
                c.res_q = a.res_q;
                c.racy = a.racy;
                c.late = late;
                c.rp_n = nullptr;
                if (a.racy && !late) {
                    // early racy sweeps: every vertex reads and updates the live volumes
                    c.volc = vb[0];
                    c.volw = vb[0];
                    c.mv_u = a.mv_u + cb;
                    c.mv_c = a.mv_c + cb;
                    c.nmv = a.nmv + par * a.ncol + k;
                } else if (!late) {
                    c.volc = vb[t & 1];
                    c.volw = vb[(t + 1) & 1];
                    c.mv_u = a.mv_u + cb;
                    c.mv_c = a.mv_c + cb;
                    c.nmv = a.nmv + par * a.ncol + k;
                } else {
                    c.volc = vb[t & 1];
                    c.volw = vb[t & 1];
                    c.cand_u = a.mv_u + cb;
                    c.cand_c = a.mv_c + cb;
                    c.cand_d = a.cd + cb;
                    c.cand_wd = a.cwd + cb;
                    c.cand_wc = a.cwc + cb;
                    c.ncand = a.ncand + k;
                }
            }
            __syncthreads();
            const int32_t nb2 = *sh.nb2;
            if (!late && !a.racy && prev_k >= 0) {
                // replay the previous class's moves into this class's write buffer
                const int64_t pa = a.class_off[(int64_t)prev_k * NBINS];
                const int64_t nr = (int64_t)__ldcg(a.nmv + prev_par * a.ncol + prev_k);
                for (int64_t i = gtid; i < nr; i += gthreads) {
                    const int32_t u = a.mv_u[pa + i];
                    const int64_t vu = a.g.vol[u];
                    vol_add(c.volw, a.mv_c[pa + i], -vu);
                    vol_add(c.volw, a.zeta[u], vu);
                }
            }
            const bool timed = a.stage_ns && tm.rank == 0 && threadIdx.x == 0;
            const uint64_t t0 = timed ? global_ns() : 0;
            // a block walks several items; the barrier keeps one item's warps
            // out of the shared tables of the next.  The first pass hands out
            // items from the end: hub chunks first, so that the hubs' decide
            // slices find their tables complete, then blocks, then the lane
            // groups; later passes alternate direction (serpentine_item).
            const int64_t step = (int64_t)sw * a.ncol + k;
            unsigned long long *smx = a.stage_max ? a.stage_max + STAGE_SLOTS * step : nullptr;
            for (int32_t p = 0; (int64_t)p * tm.size < c.bend[5]; p++) {
                const int32_t item = serpentine_item(p, tm.rank, tm.size, c.bend[5]);
                if (item < 0) continue;
                const uint64_t ti = smx && threadIdx.x == 0 ? global_ns() : 0;
                if (smx && threadIdx.x == 0 && p == 0) atomicMax(smx + ST_FIRST_ITEM, ti);
                run_item<WK, BIG, false>(c, item, sh.smem, sh.best, sh.cand, sh.last);
                __syncthreads();
                if (smx && threadIdx.x == 0)
                    atomicMax(smx + (item < c.bend[2] ? ST_GROUP : item < c.bend[4] ? ST_BLOCK : ST_CHUNK),
                              global_ns() - ti);
            }
            if (smx && threadIdx.x == 0) atomicMax(smx + ST_ITEMS_END, global_ns());
            if (nb2 > 0) {
                if (!decide_pool<WK, BIG, false>(tm, c, nb2, sh, smx)) return false;
            }
            if (smx && threadIdx.x == 0) atomicMax(smx + ST_DECIDE_END, global_ns());
            if (late || c.nrelax > 0) {
                // the block that finishes the class last re-checks its wanted
                // moves (late sweeps) or writes the hubs' deferred labels
                const bool finisher = class_finisher(a, tm, fin_base, sh.last);
                if (finisher) {
                    if (!late) {
                        apply_deferred_labels(c);
                    } else if (__ldcg(c.ncand) != 0) {
                        const uint64_t r0 = a.stage_ns ? global_ns() : 0;
                        RecheckArgs ra{c.cand_u, c.cand_c, c.cand_d, c.cand_wd, c.cand_wc, c.ncand, a.zeta,
                                       a.g.vol, c.volw, 2 * a.g.W, a.res_p, a.res_q, a.tmp_a, a.tmp_b, a.ubits,
                                       a.rc_u, a.rc_cd, a.rc_vu, a.rc_dw, c.cnt,
                                       a.g.rp, a.cstamp, sw * a.ncol + k + 1, a.stage_ns, a.racy, a.g.col};
                        recheck_block<BIG>(ra, sh.smem);
                        if (a.stage_ns && threadIdx.x == 0) atomicAdd(a.stage_ns + 2, global_ns() - r0);
                    }
                    if (smx && threadIdx.x == 0) atomicMax(smx + ST_FINISH_END, global_ns());
                }
            }
            if (!late && !a.racy) {
                prev_k = k;
                prev_par = par;
                t++;
            }
            if (!team_sync(tm, sh.gen, sh.ok)) return false;
            if (timed) a.stage_ns[0] += global_ns() - t0;
            if (tracer) {
                a.class_ns[1 + (int64_t)sw * a.ncol + k] = global_ns();
                smx[ST_MOVES] = late ? __ldcg(a.ncand + k) : __ldcg(a.nmv + par * a.ncol + k);
            }
        }
        // the sweep's counters are complete once every block has added its sums
        flush_counters(sh.bcnt, a.cnt + sw);
        if (!team_sync(tm, sh.gen, sh.ok)) return false;
        if (__ldcg(&a.cnt[sw].wanted) == 0) {
            conv = 1;
            sw++;
            break;
        }
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
        a.result[0] = sw;
        a.result[1] = conv;
        a.result[2] = (int32_t)(t & 1);   // buffer holding the final volumes
    }
    return true;
}

// ---------------------------------------------------------------------------
// PLP (Algorithm 1) of one graph, run by one team: iterations while more than
// theta labels changed.  Returns false when a barrier failed.
// ---------------------------------------------------------------------------
template <int WK, bool BIG>
__device__ bool plp_body(const PhaseArgs &a, const Team &tm, const BlockShared<PlpBest> &sh, int32_t *gt_keys,
                         void *gt_vals) {
    SweepCtx &c = *sh.c;
    int32_t it = 0;
    unsigned long long updated = (unsigned long long)a.g.n;
    unsigned long long fin_base = 0;   // same in every block of the team
    while ((double)updated > a.theta && it < a.max_iters) {
        const uint32_t salt = plp_salt_dev(a.seed, it);
        for (int32_t k = 0; k < a.ncol; k++) {
            const int64_t cb = a.class_off[(int64_t)k * NBINS], ce = a.class_off[(int64_t)k * NBINS + NBINS];
            if (ce == cb) continue;
            __syncthreads();
            if (threadIdx.x == 0) {
                *sh.nb2 = class_ctx(a, k, c);
                c.g = a.g;
                c.zeta = a.zeta;
                c.gt_keys = gt_keys;
                c.gt_vals = gt_vals;
                c.cnt = a.cnt + it;
                c.bcnt = sh.bcnt;
                c.racy = a.racy;
                c.active = a.active;
                c.tie_salt = salt;
            }
            __syncthreads();
            const int32_t nb2 = *sh.nb2;
            for (int32_t p = 0; (int64_t)p * tm.size < c.bend[5]; p++) {
                const int32_t item = serpentine_item(p, tm.rank, tm.size, c.bend[5]);
                if (item < 0) continue;
                run_item<WK, BIG, true>(c, item, sh.smem, sh.best, sh.cand, sh.last);
                __syncthreads();
            }
            if (nb2 > 0) {
                if (!decide_pool<WK, BIG, true>(tm, c, nb2, sh)) return false;
            }
            if (c.nrelax > 0 && class_finisher(a, tm, fin_base, sh.last)) apply_deferred_labels(c);
            if (!team_sync(tm, sh.gen, sh.ok)) return false;
        }
        flush_counters(sh.bcnt, a.cnt + it);
        if (!team_sync(tm, sh.gen, sh.ok)) return false;
        updated = __ldcg(&a.cnt[it].moved);
        it++;
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
        a.result[0] = it;
        a.result[1] = !((double)updated > a.theta);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Batch kernels.  The grid is cut into tiers of consecutive blocks; a tier's
// blocks form teams of team_size blocks that pull graph indices from the
// tier's queue and run each graph's phase on the team's own barrier.  A
// single graph is one tier holding one team that spans the grid.  Graphs of
// uneven size share one launch: each tier holds graphs of similar size, and
// the host sizes tiers by their share of the work.
// ---------------------------------------------------------------------------
constexpr int MAX_TIERS = 16;

struct Tier {
    int32_t begin, blocks;     // block range [begin, begin + blocks)
    int32_t team_size, team0;  // blocks per team; index of the tier's first team
    int32_t first, count;      // graphs [first, first + count) of the batch
};

struct BatchArgs {
    const PhaseArgs *graphs;   // device array, tier by tier
    int32_t *gt_keys;          // role-3b tables: GT_SLOTS per block of the grid (all -1 between uses)
    unsigned long long *gt_vals;   //   values (all 0 between uses)
    GridBarrier *bars;         // one per team
    unsigned int *queues;      // one per tier: next graph
    int32_t *team_graph;       // current graph of each team
    int32_t ntiers;
    Tier tiers[MAX_TIERS];
};

#define CD_BLOCK_SHARED(BT)                                                     \
    extern __shared__ __align__(16) unsigned char smem[];                       \
    __shared__ BT s_best[kBlock / 32];                                          \
    __shared__ unsigned s_cand, s_gen;                                          \
    __shared__ int s_last, s_ok, s_nb2;                                         \
    __shared__ long long s_grab;                                                \
    __shared__ SweepCtx s_ctx;                                                  \
    __shared__ __align__(16) unsigned long long s_args[sizeof(PhaseArgs) / 8];  \
    __shared__ unsigned long long s_bcnt[BC_N];                                 \
    if (threadIdx.x == 0) s_gen = 0;                                            \
    if (threadIdx.x < BC_N) s_bcnt[threadIdx.x] = 0;                            \
    __syncthreads();                                                            \
    const BlockShared<BT> sh{smem, s_best, &s_cand, &s_gen, &s_last, &s_ok, &s_nb2, &s_grab, &s_ctx, s_bcnt};

static_assert(sizeof(PhaseArgs) % 8 == 0, "PhaseArgs is copied in 64-bit words");

// This block's tier and team.
__device__ __forceinline__ void find_team(const BatchArgs &b, int32_t *tier, int32_t *team, Team *tm) {
    int32_t j = 0;
    while (j + 1 < b.ntiers && (int32_t)blockIdx.x >= b.tiers[j + 1].begin) j++;
    const Tier &t = b.tiers[j];
    const int32_t r = (int32_t)blockIdx.x - t.begin;
    *tier = j;
    *team = t.team0 + r / t.team_size;
    *tm = Team{r % t.team_size, t.team_size, b.bars + *team};
}

// The team's next graph (-1 when the tier's queue is empty or a barrier
// failed); its arguments are copied into shared memory.
__device__ __forceinline__ int32_t next_graph(const BatchArgs &b, int32_t tier, int32_t team, const Team &tm,
                                              unsigned *s_gen, int *s_ok, unsigned long long *s_args) {
    if (tm.rank == 0 && threadIdx.x == 0) b.team_graph[team] = (int32_t)atomicAdd(b.queues + tier, 1u);
    if (!team_sync(tm, s_gen, s_ok)) return -1;
    const int32_t q = __ldcg(b.team_graph + team);
    // every block has read the assignment before the leader can replace it
    if (!team_sync(tm, s_gen, s_ok)) return -1;
    if (q >= b.tiers[tier].count) return -1;
    const int32_t g = b.tiers[tier].first + q;
    const unsigned long long *w = reinterpret_cast<const unsigned long long *>(b.graphs + g);
    for (int i = threadIdx.x; i < (int)(sizeof(PhaseArgs) / 8); i += blockDim.x) s_args[i] = w[i];
    __syncthreads();
    return g;
}

template <int WK, bool BIG>
__global__ void __launch_bounds__(kBlock, 4) k_move_phase_batch(BatchArgs b) {
    CD_BLOCK_SHARED(PlmBest<BIG>)
    int32_t tier, team;
    Team tm;
    find_team(b, &tier, &team, &tm);
    while (next_graph(b, tier, team, tm, &s_gen, &s_ok, s_args) >= 0)
        if (!move_phase_body<WK, BIG>(*reinterpret_cast<const PhaseArgs *>(s_args), tm, sh,
                                      b.gt_keys + (size_t)blockIdx.x * GT_SLOTS,
                                      b.gt_vals + (size_t)blockIdx.x * GT_SLOTS)) return;
}

template <int WK, bool BIG>
__global__ void __launch_bounds__(kBlock, 4) k_plp_batch(BatchArgs b) {
    CD_BLOCK_SHARED(PlpBest)
    int32_t tier, team;
    Team tm;
    find_team(b, &tier, &team, &tm);
    while (next_graph(b, tier, team, tm, &s_gen, &s_ok, s_args) >= 0)
        if (!plp_body<WK, BIG>(*reinterpret_cast<const PhaseArgs *>(s_args), tm, sh,
                               b.gt_keys + (size_t)blockIdx.x * GT_SLOTS,
                               b.gt_vals + (size_t)blockIdx.x * GT_SLOTS)) return;
}

}  // namespace cd
