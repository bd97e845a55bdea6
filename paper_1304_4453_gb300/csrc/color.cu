// Distance-1 colouring used as the deterministic schedule of the move and
// label-propagation sweeps: first-fit Jones-Plassmann with hash priorities.
//
// Priority of v: (fmix32(v ^ s), v), larger wins.  Round r: every
// uncoloured vertex whose priority beats all neighbours that were uncoloured
// when the round began takes the smallest colour not used by its neighbours
// coloured in earlier rounds.  Such vertices are pairwise non-adjacent, so a
// round's outcome does not depend on processing order, and the result equals
// greedy colouring in descending priority order.
//
// state[v] = -1 while uncoloured, else (round << 32) | colour, written with a
// single 64-bit store so that a reader sees colour and round together.
// Rounds run back to back on the device (the list length lives in device
// memory); the host checks for completion every few rounds.
#include "common.cuh"

namespace cd {

__global__ void k_color_prio(int64_t n, uint32_t s, uint64_t *prio) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        prio[v] = fmix32((uint32_t)v ^ s);
}

__device__ __forceinline__ bool prio_gt(uint64_t px, int32_t x, uint64_t pv, int32_t v) {
    return px > pv || (px == pv && x > v);
}

// One warp per listed vertex.
__global__ void k_color_round(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const uint64_t *__restrict__ prio, const int32_t *__restrict__ list,
                              const unsigned long long *count_in, int32_t round, int64_t *state, int32_t *next,
                              unsigned long long *next_count) {
    const int lane = threadIdx.x & 31;
    const int64_t count = (int64_t)*count_in;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nwarps) {
        const int32_t v = list[i];
        const uint64_t pv = prio[v];
        const int64_t beg = rp[v], end = rp[v + 1];
        bool is_max = true;
        unsigned long long bits = 0;
        for (int64_t e0 = beg; e0 < end; e0 += 32) {
            const int64_t e = e0 + lane;
            if (e < end) {
                const int32_t x = col[e];
                const int64_t st = ((volatile int64_t *)state)[x];
                const bool uncol = st < 0 || (int32_t)(st >> 32) == round;
                if (uncol) {
                    if (prio_gt(prio[x], x, pv, v)) is_max = false;
                } else {
                    const uint32_t c = (uint32_t)st;
                    if (c < 64) bits |= 1ull << c;
                }
            }
            if (__any_sync(0xffffffffu, !is_max)) { is_max = false; break; }
        }
        if (!is_max) {
            if (lane == 0) next[atomicAdd(next_count, 1ull)] = v;
            continue;
        }
        for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        uint32_t c;
        if (bits != ~0ull) {
            c = __ffsll((long long)~bits) - 1;
        } else {
            // all of 0..63 taken: scan further windows of 64 colours
            uint32_t base = 64;
            while (true) {
                unsigned long long b2 = 0;
                for (int64_t e = beg + lane; e < end; e += 32) {
                    const int64_t st = state[col[e]];
                    const uint32_t cc = (uint32_t)st;
                    if (st >= 0 && cc >= base && cc < base + 64) b2 |= 1ull << (cc - base);
                }
                for (int o = 16; o > 0; o >>= 1) b2 |= __shfl_xor_sync(0xffffffffu, b2, o);
                if (b2 != ~0ull) { c = base + __ffsll((long long)~b2) - 1; break; }
                base += 64;
            }
        }
        if (lane == 0) state[v] = ((int64_t)round << 32) | (int64_t)c;
    }
}

__global__ void k_color_extract(const int64_t *state, int64_t n, int32_t *color, unsigned int *maxc) {
    unsigned int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c = (uint32_t)state[i];
        color[i] = (int32_t)c;
        m = max(m, c + 1);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxc, m);
}

int32_t color_graph(const GraphView &g, uint64_t seed, int32_t *color, cudaStream_t s) {
    if (g.n == 0) return 0;
    const uint32_t sw = seed_word(seed);
    constexpr int ROUNDS_PER_CHECK = 8;
    DBuf<int64_t> state(g.n, s);
    DBuf<uint64_t> prio(g.n, s);
    CD_CUDA(cudaMemsetAsync(state.p, 0xff, g.n * sizeof(int64_t), s));
    { k_color_prio<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(g.n, sw, prio.p); ::cd::note_launch(); }
    DBuf<int32_t> la(g.n, s), lb(g.n, s);
    iota32(la.p, g.n, s);
    DBuf<unsigned long long> cnt(2, s);   // list lengths: [0] current, [1] next
    const unsigned long long n0 = (unsigned long long)g.n;
    CD_CUDA(cudaMemcpyAsync(cnt.p, &n0, sizeof(n0), cudaMemcpyHostToDevice, s));
    Pinned h(sizeof(unsigned long long));
    int64_t known = g.n;   // upper bound on the current list length
    int32_t round = 0;
    int which = 0;         // cnt[which] holds the current length
    while (true) {
        for (int r = 0; r < ROUNDS_PER_CHECK; r++) {
            int32_t *cur = (round & 1) ? lb.p : la.p;
            int32_t *nxt = (round & 1) ? la.p : lb.p;
            CD_CUDA(cudaMemsetAsync(cnt.p + (1 - which), 0, sizeof(unsigned long long), s));
            { k_color_round<<<grid_for(known * 32, kBlock, 152 * 64), kBlock, 0, s>>>(
                  g.rp, g.col, prio.p, cur, cnt.p + which, round, state.p, nxt, cnt.p + (1 - which)); ::cd::note_launch(); }
            CD_LAUNCH_CHECK();
            which = 1 - which;
            round++;
        }
        CD_CUDA(cudaMemcpyAsync(h.p, cnt.p + which, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        const int64_t left = (int64_t)*h.as<unsigned long long>();
        if (left == 0) break;
        if (left >= known) raise(CD_ECUDA, "colouring made no progress by round %d", round);
        known = left;
    }
    DBuf<unsigned int> maxc(1, s);
    maxc.zero();
    { k_color_extract<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(state.p, g.n, color, maxc.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned hm(sizeof(unsigned int));
    CD_CUDA(cudaMemcpyAsync(hm.p, maxc.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return (int32_t)*hm.as<unsigned int>();
}

}  // namespace cd
