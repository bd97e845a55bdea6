// Distance-1 colouring used as the deterministic schedule of the move and
// label-propagation sweeps: first-fit Jones-Plassmann with hash priorities.
//
// Priority of v: (fmix32(v ^ s), v), larger wins.  Jones-Plassmann colours a
// vertex once all of its higher-priority neighbours are coloured, giving it
// the smallest colour none of them uses; the result equals greedy colouring
// in descending priority order.
//
// Dependency-count form: wait[v] = number of higher-priority neighbours.
// Vertices with wait 0 form the first frontier.  A frontier vertex reads the
// colours of its higher-priority neighbours (all set), takes the smallest
// free colour, and decrements wait of its lower-priority neighbours; those
// that reach 0 form the next frontier.  Every adjacency entry is read once to
// count and once when its row's vertex is coloured (plus a rescan per extra
// window of 64 colours).  Frontier vertices of degree <= 64 are handled by one
// warp each, up to 4096 by one block each, and the adjacency of larger ones
// is cut into chunks spread over all blocks (k_color_round_hubs): a round
// lasts as long as its slowest vertex.  Rounds run back to back on
// the device (frontier lengths live in device memory); the host checks for
// completion every few rounds.
#include "common.cuh"

namespace cd {

constexpr int COLOR_WARP_DEG = 64;     // frontier vertices up to this degree: one warp each
constexpr int COLOR_BIG_DEG = 4096;    // up to this degree: one block each; above: chunked

__device__ __forceinline__ bool prio_gt(uint32_t hx, int32_t x, uint32_t hv, int32_t v) {
    return hx > hv || (hx == hv && x > v);
}

// Next-round frontier: three lists by degree (warp / block / chunked).
struct Frontier {
    int32_t *list[3];
    unsigned long long *count[3];
};

__device__ __forceinline__ void push_ready(int32_t x, const int64_t *rp, const Frontier &f) {
    const int64_t d = rp[x + 1] - rp[x];
    const int t = d <= COLOR_WARP_DEG ? 0 : d <= COLOR_BIG_DEG ? 1 : 2;
    f.list[t][atomicAdd(f.count[t], 1ull)] = x;
}

// wait[v] and the first frontier; one warp per vertex.
__global__ void k_color_init(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int64_t n, uint32_t s,
                             uint32_t *hash, int32_t *wait, int32_t *color, Frontier nf, int32_t *hub_slot,
                             unsigned int *nhubs) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const uint32_t hv = fmix32((uint32_t)v ^ s);
        const int64_t beg = rp[v], end = rp[v + 1];
        int cnt = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t x = col[e];
            cnt += prio_gt(fmix32((uint32_t)x ^ s), x, hv, (int32_t)v) ? 1 : 0;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            hash[v] = hv;
            wait[v] = cnt;
            color[v] = -1;
            if (end - beg > COLOR_BIG_DEG) hub_slot[v] = (int32_t)atomicAdd(nhubs, 1u);
            if (cnt == 0) push_ready((int32_t)v, rp, nf);
        }
    }
}

// Colours of higher-priority neighbours falling in [base, base + 64).
__device__ __forceinline__ unsigned long long window_bits(const int64_t *rp, const int32_t *col, const uint32_t *hash,
                                                          const int32_t *color, int32_t v, uint32_t hv, int64_t e0,
                                                          int64_t step, uint32_t base) {
    unsigned long long b = 0;
    for (int64_t e = rp[v] + e0; e < rp[v + 1]; e += step) {
        const int32_t x = col[e];
        if (prio_gt(hash[x], x, hv, v)) {
            const uint32_t c = (uint32_t)color[x];
            if (c >= base && c < base + 64) b |= 1ull << (c - base);
        }
    }
    return b;
}

// One warp per frontier vertex (degree <= COLOR_BIG_DEG).
__global__ void k_color_round_warp(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                   const uint32_t *__restrict__ hash, const int32_t *list,
                                   const unsigned long long *count_in, int32_t *wait, int32_t *color, Frontier nf,
                                   unsigned long long *done) {
    __shared__ int64_t s_count;
    const int lane = threadIdx.x & 31;
    // one read of the frontier length per block: every warp reading it would
    // queue thousands of requests on one L2 line
    if (threadIdx.x == 0) s_count = (int64_t)*count_in;
    __syncthreads();
    const int64_t count = s_count;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < count; i += nwarps) {
        const int32_t v = list[i];
        const uint32_t hv = hash[v];
        const int64_t beg = rp[v], end = rp[v + 1];
        unsigned long long bits = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t x = col[e];
            if (prio_gt(hash[x], x, hv, v)) {
                const uint32_t c = (uint32_t)color[x];
                if (c < 64) bits |= 1ull << c;
            } else if (atomicSub(&wait[x], 1) == 1) {
                push_ready(x, rp, nf);
            }
        }
        for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        uint32_t base = 0;
        while (bits == ~0ull) {
            base += 64;
            bits = window_bits(rp, col, hash, color, v, hv, lane, 32, base);
            for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        }
        if (lane == 0) {
            color[v] = (int32_t)(base + __ffsll((long long)~bits) - 1);
            atomicAdd(done, 1ull);
        }
    }
}

// One block per frontier vertex (COLOR_WARP_DEG < degree <= COLOR_BIG_DEG).
__global__ void k_color_round_block(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                    const uint32_t *__restrict__ hash, const int32_t *list,
                                    const unsigned long long *count_in, int32_t *wait, int32_t *color, Frontier nf,
                                    unsigned long long *done) {
    __shared__ unsigned long long sbits;
    __shared__ int64_t s_count;
    if (threadIdx.x == 0) s_count = (int64_t)*count_in;
    __syncthreads();
    const int64_t count = s_count;
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t v = list[i];
        const uint32_t hv = hash[v];
        const int64_t beg = rp[v], end = rp[v + 1];
        if (threadIdx.x == 0) sbits = 0;
        __syncthreads();
        unsigned long long bits = 0;
        for (int64_t e = beg + threadIdx.x; e < end; e += kBlock) {
            const int32_t x = col[e];
            if (prio_gt(hash[x], x, hv, v)) {
                const uint32_t c = (uint32_t)color[x];
                if (c < 64) bits |= 1ull << c;
            } else if (atomicSub(&wait[x], 1) == 1) {
                push_ready(x, rp, nf);
            }
        }
        for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        if ((threadIdx.x & 31) == 0) atomicOr(&sbits, bits);
        __syncthreads();
        bits = sbits;
        uint32_t base = 0;
        while (bits == ~0ull) {
            base += 64;
            __syncthreads();
            if (threadIdx.x == 0) sbits = 0;
            __syncthreads();
            unsigned long long b = window_bits(rp, col, hash, color, v, hv, threadIdx.x, kBlock, base);
            for (int o = 16; o > 0; o >>= 1) b |= __shfl_xor_sync(0xffffffffu, b, o);
            if ((threadIdx.x & 31) == 0) atomicOr(&sbits, b);
            __syncthreads();
            bits = sbits;
        }
        if (threadIdx.x == 0) {
            color[v] = (int32_t)(base + __ffsll((long long)~bits) - 1);
            atomicAdd(done, 1ull);
        }
        __syncthreads();
    }
}

// Frontier hubs (degree > COLOR_BIG_DEG): each hub's adjacency is cut into
// chunks of COLOR_CHUNK entries, and the (hub, chunk) items of the round are
// spread over all blocks.  A chunk ORs the colours (< COLOR_BITS) of its
// higher-priority neighbours into the hub's bitmap and releases its
// lower-priority neighbours; the last chunk of a hub takes the first free
// colour (scanning the adjacency for windows beyond COLOR_BITS if needed).
constexpr int COLOR_CHUNK = 2048;
constexpr int COLOR_BITS = 4096;
constexpr int COLOR_WORDS = COLOR_BITS / 32;

__global__ void k_color_round_hubs(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                   const uint32_t *__restrict__ hash, const int32_t *list,
                                   const unsigned long long *count_in, const int32_t *hub_slot, uint32_t *bitmaps,
                                   unsigned int *chunks_done, int32_t *wait, int32_t *color, Frontier nf,
                                   unsigned long long *done) {
    __shared__ uint32_t sbm[COLOR_WORDS];
    __shared__ int s_last;
    __shared__ unsigned long long sbits;
    __shared__ int64_t s_count;
    if (threadIdx.x == 0) s_count = (int64_t)*count_in;
    __syncthreads();
    const int64_t count = s_count;
    int64_t item0 = 0;
    for (int64_t i = 0; i < count; i++) {
        const int32_t v = list[i];
        const int64_t beg = rp[v], end = rp[v + 1];
        const int64_t nch = (end - beg + COLOR_CHUNK - 1) / COLOR_CHUNK;
        const uint32_t hv = hash[v];
        const int32_t slot = hub_slot[v];
        uint32_t *bm = bitmaps + (size_t)slot * COLOR_WORDS;
        // items item0 .. item0 + nch - 1 belong to this hub
        int64_t first = item0 + ((blockIdx.x - item0 % gridDim.x) + gridDim.x) % gridDim.x;
        for (int64_t it = first; it < item0 + nch; it += gridDim.x) {
            const int64_t j = it - item0;
            for (int w = threadIdx.x; w < COLOR_WORDS; w += kBlock) sbm[w] = 0;
            __syncthreads();
            const int64_t cb = beg + j * COLOR_CHUNK, ce = min(end, cb + COLOR_CHUNK);
            for (int64_t e = cb + threadIdx.x; e < ce; e += kBlock) {
                const int32_t x = col[e];
                if (prio_gt(hash[x], x, hv, v)) {
                    const uint32_t c = (uint32_t)color[x];
                    if (c < COLOR_BITS) atomicOr(&sbm[c >> 5], 1u << (c & 31));
                } else if (atomicSub(&wait[x], 1) == 1) {
                    push_ready(x, rp, nf);
                }
            }
            __syncthreads();
            for (int w = threadIdx.x; w < COLOR_WORDS; w += kBlock)
                if (sbm[w]) atomicOr(&bm[w], sbm[w]);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(&chunks_done[slot], 1u) == (unsigned)(nch - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                // first zero bit of the bitmap
                if (threadIdx.x == 0) sbits = ~0ull;
                __syncthreads();
                for (int w = threadIdx.x; w < COLOR_WORDS; w += kBlock) {
                    const uint32_t word = __ldcg(bm + w);
                    if (word != 0xffffffffu) atomicMin(&sbits, (unsigned long long)(w * 32 + __ffs(~word) - 1));
                }
                __syncthreads();
                uint32_t c = (uint32_t)sbits;
                if (sbits == ~0ull) {
                    // every colour below COLOR_BITS is taken: scan windows of 64 above it
                    uint32_t base = COLOR_BITS;
                    while (true) {
                        __syncthreads();
                        if (threadIdx.x == 0) sbits = 0;
                        __syncthreads();
                        unsigned long long b = window_bits(rp, col, hash, color, v, hv, threadIdx.x, kBlock, base);
                        for (int o = 16; o > 0; o >>= 1) b |= __shfl_xor_sync(0xffffffffu, b, o);
                        if ((threadIdx.x & 31) == 0) atomicOr(&sbits, b);
                        __syncthreads();
                        const unsigned long long bits = sbits;
                        if (bits != ~0ull) { c = base + __ffsll((long long)~bits) - 1; break; }
                        base += 64;
                    }
                }
                if (threadIdx.x == 0) {
                    color[v] = (int32_t)c;
                    atomicAdd(done, 1ull);
                }
            }
            __syncthreads();
        }
        item0 += nch;
    }
}

__global__ void k_color_max(const int32_t *color, int64_t n, unsigned int *maxc) {
    unsigned int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned int)color[i] + 1);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxc, m);
}

int32_t color_graph(const GraphView &g, uint64_t seed, int32_t *color, cudaStream_t s) {
    if (g.n == 0) return 0;
    const uint32_t sw = seed_word(seed);
    constexpr int ROUNDS_PER_CHECK = 8;
    DBuf<uint32_t> hash(g.n, s);
    DBuf<int32_t> wait(g.n, s);
    DBuf<int32_t> lists(6 * g.n, s);          // three tiers, current and next
    DBuf<unsigned long long> cnt(7, s);       // [tier * 2 + side], [6] coloured
    cnt.zero();
    Frontier F[2];
    for (int side = 0; side < 2; side++)
        for (int t = 0; t < 3; t++) {
            F[side].list[t] = lists.p + (size_t)(2 * t + side) * g.n;
            F[side].count[t] = cnt.p + 2 * t + side;
        }
    // every chunked hub has more than COLOR_BIG_DEG entries
    const int64_t max_hubs = g.nnz / (COLOR_BIG_DEG + 1) + 1;
    DBuf<int32_t> hub_slot(g.n, s);
    DBuf<uint32_t> bitmaps((size_t)max_hubs * COLOR_WORDS, s);
    DBuf<unsigned int> chunks_done(max_hubs, s), nhubs(1, s);
    bitmaps.zero();
    chunks_done.zero();
    nhubs.zero();
    { k_color_init<<<grid_for(g.n * 32, kBlock, 152 * 64), kBlock, 0, s>>>(g.rp, g.col, g.n, sw, hash.p, wait.p, color,
                                                                          F[0], hub_slot.p, nhubs.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned h(sizeof(unsigned long long));
    int cur = 0;
    int64_t rounds = 0;
    while (true) {
        for (int r = 0; r < ROUNDS_PER_CHECK; r++) {
            const int nx = 1 - cur;
            for (int t = 0; t < 3; t++) CD_CUDA(cudaMemsetAsync(F[nx].count[t], 0, sizeof(unsigned long long), s));
            { k_color_round_warp<<<152 * 4, kBlock, 0, s>>>(g.rp, g.col, hash.p, F[cur].list[0], F[cur].count[0],
                                                          wait.p, color, F[nx], cnt.p + 6); ::cd::note_launch(); }
            { k_color_round_block<<<152 * 4, kBlock, 0, s>>>(g.rp, g.col, hash.p, F[cur].list[1], F[cur].count[1],
                                                           wait.p, color, F[nx], cnt.p + 6); ::cd::note_launch(); }
            { k_color_round_hubs<<<152 * 2, kBlock, 0, s>>>(g.rp, g.col, hash.p, F[cur].list[2], F[cur].count[2],
                                                          hub_slot.p, bitmaps.p, chunks_done.p, wait.p, color, F[nx],
                                                          cnt.p + 6); ::cd::note_launch(); }
            CD_LAUNCH_CHECK();
            cur = nx;
            rounds++;
        }
        CD_CUDA(cudaMemcpyAsync(h.p, cnt.p + 6, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        const int64_t coloured = (int64_t)*h.as<unsigned long long>();
        if (coloured >= g.n) break;
        // every round colours at least one vertex
        if (rounds > g.n + 64) raise(CD_ECUDA, "colouring did not finish after %lld rounds", (long long)rounds);
    }
    DBuf<unsigned int> maxc(1, s);
    maxc.zero();
    { k_color_max<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(color, g.n, maxc.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned hm(sizeof(unsigned int));
    CD_CUDA(cudaMemcpyAsync(hm.p, maxc.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return (int32_t)*hm.as<unsigned int>();
}

}  // namespace cd
