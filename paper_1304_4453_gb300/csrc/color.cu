// Distance-1 colouring used as the deterministic schedule of the move and
// label-propagation sweeps: first-fit Jones-Plassmann with hash priorities.
//
// Round r: every uncoloured vertex whose priority (fmix32(v ^ s), v) beats
// all neighbours that were uncoloured when the round began takes the
// smallest colour not used by its neighbours coloured in earlier rounds.
// Such vertices are pairwise non-adjacent, so the outcome of a round does
// not depend on the order in which they are processed.
//
// state[v] = -1 while uncoloured, else (round << 32) | colour, written with a
// single 64-bit store so that a reader sees colour and round together.
#include "common.cuh"

namespace cd {

__device__ __forceinline__ bool prio_gt(uint32_t hx, int32_t x, uint32_t hv, int32_t v) {
    return hx > hv || (hx == hv && x > v);
}

// One warp per listed vertex.
__global__ void k_color_round(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const int32_t *__restrict__ list, int64_t count, uint32_t s, int32_t round,
                              int64_t *state, int32_t *next, unsigned long long *next_count) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nwarps) {
        int32_t v = list[i];
        uint32_t hv = fmix32((uint32_t)v ^ s);
        int64_t beg = rp[v], end = rp[v + 1];
        bool is_max = true;
        unsigned long long bits = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            int32_t x = col[e];
            int64_t st = ((volatile int64_t *)state)[x];
            bool uncol = st < 0 || (int32_t)(st >> 32) == round;
            if (uncol) {
                if (prio_gt(fmix32((uint32_t)x ^ s), x, hv, v)) is_max = false;
            } else {
                uint32_t c = (uint32_t)st;
                if (c < 64) bits |= 1ull << c;
            }
        }
        is_max = __all_sync(0xffffffffu, is_max);
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
                    int64_t st = state[col[e]];
                    uint32_t cc = (uint32_t)st;
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
    DBuf<int64_t> state(g.n, s);
    CD_CUDA(cudaMemsetAsync(state.p, 0xff, g.n * sizeof(int64_t), s));
    DBuf<int32_t> la(g.n, s), lb(g.n, s);
    iota32(la.p, g.n, s);
    DBuf<unsigned long long> cnt(1, s);
    Pinned h(sizeof(unsigned long long));
    int64_t count = g.n;
    int32_t round = 0;
    while (count > 0) {
        cnt.zero();
        k_color_round<<<grid_for(count * 32, kBlock, 152 * 64), kBlock, 0, s>>>(g.rp, g.col, la.p, count, sw, round,
                                                                               state.p, lb.p, cnt.p);
        CD_LAUNCH_CHECK();
        CD_CUDA(cudaMemcpyAsync(h.p, cnt.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        int64_t left = (int64_t)*h.as<unsigned long long>();
        if (left >= count) raise(CD_ECUDA, "colouring made no progress in round %d", round);
        count = left;
        std::swap(la, lb);
        round++;
    }
    DBuf<unsigned int> maxc(1, s);
    maxc.zero();
    k_color_extract<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(state.p, g.n, color, maxc.p);
    CD_LAUNCH_CHECK();
    Pinned hm(sizeof(unsigned int));
    CD_CUDA(cudaMemcpyAsync(hm.p, maxc.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return (int32_t)*hm.as<unsigned int>();
}

}  // namespace cd
