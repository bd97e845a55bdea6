// Colouring used as the deterministic schedule of the move and label-
// propagation sweeps: first-fit Jones-Plassmann with hash priorities on the
// graph without its hub-hub edges (hubs: more than HUB_RELAX neighbours).
//
// Priority of v: (fmix32(v ^ s), v), larger wins.  Jones-Plassmann colours a
// vertex once all of its higher-priority neighbours are coloured, giving it
// the smallest colour none of them uses; the result equals greedy colouring
// in descending priority order.  A hub neither waits for nor avoids the
// colours of its hub neighbours.
//
// Dependency-count form: wait[v] = number of higher-priority neighbours.
// Vertices with wait 0 form the first frontier.  A frontier vertex reads the
// colours of its higher-priority neighbours (all set), takes the smallest
// free colour, and decrements wait of its lower-priority neighbours; those
// that reach 0 form the next frontier.  Every adjacency entry is read once to
// count and once when its row's vertex is coloured (plus a rescan per extra
// window of 64 colours).  Frontier vertices of degree <= 32 are handled by one
// warp each, up to 256 by one block each, and the adjacency of larger ones
// is cut into chunks of 256 entries spread over all blocks
// (color_chunk_items): a round lasts as long as its slowest vertex, so no
// thread walks more than a few entries of one vertex.  All rounds run inside one persistent
// cooperative kernel, separated by a grid barrier; the frontiers rotate over
// three buffers so that the buffer a round pushes into was cleared a round
// earlier, and the kernel stops at the first round whose frontier is empty.
#include <algorithm>

#include "barrier.cuh"

namespace cd {

constexpr int COLOR_WARP_DEG = 32;     // frontier vertices up to this degree: one warp each (R-MAT 22: 64 -> 32
                                       // took the colouring from 111 to 104 ms per run; 128 was slower)
constexpr int COLOR_BIG_DEG = 256;     // up to this degree: one block each; above: chunked (R-MAT 22: 1024 -> 256
                                       // took the colouring from 122 to 112 ms per run)
constexpr int COLOR_CHUNK = 256;       // adjacency entries per chunk item (R-MAT 22: 1024 -> 256 took the
                                       // colouring from 143.6 to 127.0 ms per run; 128 and 64 were slower)
static_assert(COLOR_WARP_DEG <= COLOR_BIG_DEG && COLOR_BIG_DEG <= HUB_RELAX,
              "warp- and block-tier vertices are never hubs");

__device__ __forceinline__ bool prio_gt(uint32_t hx, int32_t x, uint32_t hv, int32_t v) {
    return hx > hv || (hx == hv && x > v);
}

// Next-round frontier: vertex lists of the warp and block tiers, and the
// chunk items (vertex | chunk << 32) of the larger vertices.
struct Frontier {
    int32_t *list[2];
    unsigned long long *items;
    unsigned long long *count[3];   // warp, block, chunk items
};

__device__ __forceinline__ int64_t colour_chunks(int64_t deg) { return (deg + COLOR_CHUNK - 1) / COLOR_CHUNK; }

__device__ __forceinline__ void push_ready(int32_t x, const int64_t *rp, const Frontier &f) {
    const int64_t d = rp[x + 1] - rp[x];
    if (d <= COLOR_BIG_DEG) {
        const int t = d <= COLOR_WARP_DEG ? 0 : 1;
        f.list[t][atomicAdd(f.count[t], 1ull)] = x;
    } else {
        const int64_t nch = colour_chunks(d);
        const unsigned long long b = atomicAdd(f.count[2], (unsigned long long)nch);
        for (int64_t j = 0; j < nch; j++) f.items[b + j] = (unsigned long long)(uint32_t)x | ((unsigned long long)j << 32);
    }
}

// wait[v] and the first frontier; one warp per vertex.
__global__ void k_color_init(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int64_t n, uint32_t s,
                             uint32_t *hash, int32_t *wait, int32_t *color, Frontier nf, int32_t *chunk_slot,
                             unsigned int *nchunked) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const uint32_t hv = fmix32((uint32_t)v ^ s);
        const int64_t beg = rp[v], end = rp[v + 1];
        const bool vh = end - beg > HUB_RELAX;
        int cnt = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t x = col[e];
            if (vh && relaxed_hub(rp, x)) continue;
            cnt += prio_gt(fmix32((uint32_t)x ^ s), x, hv, (int32_t)v) ? 1 : 0;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            hash[v] = hv;
            wait[v] = cnt;
            color[v] = -1;
            if (end - beg > COLOR_BIG_DEG) chunk_slot[v] = (int32_t)atomicAdd(nchunked, 1u);
            if (cnt == 0) push_ready((int32_t)v, rp, nf);
        }
    }
}

// Colours of higher-priority neighbours falling in [base, base + 64)
// (hub neighbours of a hub excluded).
__device__ __forceinline__ unsigned long long window_bits(const int64_t *rp, const int32_t *col, const uint32_t *hash,
                                                          const int32_t *color, int32_t v, uint32_t hv, int64_t e0,
                                                          int64_t step, uint32_t base, bool vh) {
    unsigned long long b = 0;
    for (int64_t e = rp[v] + e0; e < rp[v + 1]; e += step) {
        const int32_t x = col[e];
        if (vh && relaxed_hub(rp, x)) continue;
        if (prio_gt(hash[x], x, hv, v)) {
            const uint32_t c = (uint32_t)color[x];
            if (c >= base && c < base + 64) b |= 1ull << (c - base);
        }
    }
    return b;
}

// One warp per frontier vertex (degree <= COLOR_WARP_DEG).
__device__ __forceinline__ void color_warp_items(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                 const uint32_t *__restrict__ hash, const int32_t *list,
                                                 int64_t count, int32_t *wait, int32_t *color, const Frontier &nf,
                                                 unsigned long long *done) {
    const int lane = threadIdx.x & 31;
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
            bits = window_bits(rp, col, hash, color, v, hv, lane, 32, base, false);   // degree <= 32: no hub
            for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        }
        if (lane == 0) {
            color[v] = (int32_t)(base + __ffsll((long long)~bits) - 1);
            atomicAdd(done, 1ull);
        }
    }
}

// One thread's share of a frontier vertex's adjacency [beg, end), stride
// `step`: higher-priority neighbours contribute their colour (below NB, into
// the returned bits, or into the shared bitmap `sbm` when NB > 64), and
// lower-priority neighbours are released (the last one pushes itself).  Four
// entries are loaded per step before any is used, so a thread keeps several
// loads in flight.
template <int NB>
__device__ __forceinline__ unsigned long long scan_neighbours(const int64_t *__restrict__ rp,
                                                              const int32_t *__restrict__ col,
                                                              const uint32_t *__restrict__ hash, int32_t *wait,
                                                              int32_t *color, const Frontier &nf, int32_t v,
                                                              uint32_t hv, bool vh, int64_t beg, int64_t end,
                                                              int64_t first, int64_t step, uint32_t *sbm) {
    constexpr int U = 4;
    unsigned long long bits = 0;
    for (int64_t e0 = beg + first; e0 < end; e0 += step * U) {
        int32_t x[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t e = e0 + u * step;
            ok[u] = e < end;
            x[u] = ok[u] ? col[e] : 0;
        }
        if (vh) {
#pragma unroll
            for (int u = 0; u < U; u++) ok[u] = ok[u] && !relaxed_hub(rp, x[u]);
        }
        uint32_t hx[U];
#pragma unroll
        for (int u = 0; u < U; u++) hx[u] = ok[u] ? hash[x[u]] : 0u;
        bool hi[U];
#pragma unroll
        for (int u = 0; u < U; u++) hi[u] = ok[u] && prio_gt(hx[u], x[u], hv, v);
        int32_t cx[U];
#pragma unroll
        for (int u = 0; u < U; u++) cx[u] = hi[u] ? color[x[u]] : -1;
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (hi[u]) {
                const uint32_t c = (uint32_t)cx[u];
                if (NB == 64) {
                    if (c < 64) bits |= 1ull << c;
                } else if (c < (uint32_t)NB) {
                    atomicOr(&sbm[c >> 5], 1u << (c & 31));
                }
            } else if (ok[u] && atomicSub(&wait[x[u]], 1) == 1) {
                push_ready(x[u], rp, nf);
            }
        }
    }
    return bits;
}

// One block per frontier vertex (COLOR_WARP_DEG < degree <= COLOR_BIG_DEG).
__device__ __forceinline__ void color_block_items(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                  const uint32_t *__restrict__ hash, const int32_t *list,
                                                  int64_t count, int32_t *wait, int32_t *color, const Frontier &nf,
                                                  unsigned long long *done, unsigned long long &sbits) {
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t v = list[i];
        const uint32_t hv = hash[v];
        const int64_t beg = rp[v], end = rp[v + 1];
        const bool vh = end - beg > HUB_RELAX;
        if (threadIdx.x == 0) sbits = 0;
        __syncthreads();
        const unsigned long long bits0 = scan_neighbours<64>(rp, col, hash, wait, color, nf, v, hv, vh, beg, end,
                                                              threadIdx.x, kBlock, nullptr);
        unsigned long long bits = bits0;
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
            unsigned long long b = window_bits(rp, col, hash, color, v, hv, threadIdx.x, kBlock, base, vh);
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

// Frontier vertices above COLOR_BIG_DEG: each one's adjacency is cut into
// chunks of COLOR_CHUNK entries, queued as (vertex, chunk) items when the
// vertex was released, and the items of the round are spread over all
// blocks.  A chunk ORs the colours (< COLOR_BITS) of its higher-priority
// neighbours into the vertex's bitmap and releases its lower-priority
// neighbours; the last chunk of a vertex takes the first free colour
// (scanning the adjacency for windows beyond COLOR_BITS if needed).
constexpr int COLOR_BITS = 4096;
constexpr int COLOR_WORDS = COLOR_BITS / 32;

struct ChunkShared {
    uint32_t sbm[COLOR_WORDS];
    int last;
};

__device__ __forceinline__ void color_chunk_items(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                  const uint32_t *__restrict__ hash, const unsigned long long *items,
                                                  int64_t count, const int32_t *chunk_slot, uint32_t *bitmaps,
                                                  unsigned int *chunks_done, int32_t *wait, int32_t *color,
                                                  const Frontier &nf, unsigned long long *done, ChunkShared &hs,
                                                  unsigned long long &sbits) {
    uint32_t *sbm = hs.sbm;
    int &s_last = hs.last;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        const unsigned long long item = items[it];
        const int32_t v = (int32_t)(item & 0xffffffffull);
        const int64_t j = (int64_t)(item >> 32);
        const int64_t beg = rp[v], end = rp[v + 1];
        const int64_t nch = colour_chunks(end - beg);
        const bool vh = end - beg > HUB_RELAX;
        const uint32_t hv = hash[v];
        const int32_t slot = chunk_slot[v];
        uint32_t *bm = bitmaps + (size_t)slot * COLOR_WORDS;
        for (int w = threadIdx.x; w < COLOR_WORDS; w += kBlock) sbm[w] = 0;
        __syncthreads();
        const int64_t cb = beg + j * COLOR_CHUNK, ce = min(end, cb + COLOR_CHUNK);
        scan_neighbours<COLOR_BITS>(rp, col, hash, wait, color, nf, v, hv, vh, cb, ce, threadIdx.x, kBlock, sbm);
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
                    unsigned long long b = window_bits(rp, col, hash, color, v, hv, threadIdx.x, kBlock, base, vh);
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
}

__global__ void k_color_max(const int32_t *color, int64_t n, unsigned int *maxc) {
    unsigned int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned int)color[i] + 1);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxc, m);
}

// Every round of the colouring in one cooperative launch.  Frontier side r%3
// is read in round r, side (r+1)%3 receives the next frontier, and block 0
// clears side (r+2)%3, which round r-1 read and round r+1 fills.  All blocks
// leave together at the first round whose frontier is empty (every vertex is
// coloured then), or after max_rounds rounds.
struct ColorArgs {
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *hash;
    int64_t n;
    int32_t *wait, *color;
    int32_t *lists;                // [3 sides][2 tiers][n]
    unsigned long long *items;     // [3 sides][icap] chunk items
    int64_t icap;
    unsigned long long *counts;    // [3 sides][3 tiers]
    unsigned long long *done;
    const int32_t *chunk_slot;
    uint32_t *bitmaps;
    unsigned int *chunks_done;
    GridBarrier *bar;
    int64_t max_rounds;
    int64_t *rounds;               // out: rounds run
};

__device__ __forceinline__ Frontier frontier_side(const ColorArgs &a, int side) {
    Frontier f;
    for (int t = 0; t < 2; t++) f.list[t] = a.lists + (size_t)(2 * side + t) * a.n;
    f.items = a.items + (size_t)side * a.icap;
    for (int t = 0; t < 3; t++) f.count[t] = a.counts + 3 * side + t;
    return f;
}

__global__ void __launch_bounds__(kBlock) k_color_persistent(ColorArgs a) {
    __shared__ unsigned s_gen;
    __shared__ int s_ok;
    __shared__ unsigned long long s_cnt[3];
    __shared__ unsigned long long sbits;
    __shared__ ChunkShared hs;
    const Team tm{(int32_t)blockIdx.x, (int32_t)gridDim.x, a.bar};
    if (threadIdx.x == 0) s_gen = 0;
    __syncthreads();
    int64_t r = 0;
    for (;; r++) {
        const int cur = (int)(r % 3), nx = (int)((r + 1) % 3), old = (int)((r + 2) % 3);
        if (threadIdx.x < 3) s_cnt[threadIdx.x] = __ldcg(a.counts + 3 * cur + threadIdx.x);
        if (blockIdx.x == 0 && threadIdx.x < 3) a.counts[3 * old + threadIdx.x] = 0;
        __syncthreads();
        if (s_cnt[0] + s_cnt[1] + s_cnt[2] == 0 || r >= a.max_rounds) break;
        const Frontier fc = frontier_side(a, cur), fn = frontier_side(a, nx);
        if (s_cnt[0])
            color_warp_items(a.rp, a.col, a.hash, fc.list[0], (int64_t)s_cnt[0], a.wait, a.color, fn, a.done);
        if (s_cnt[1])
            color_block_items(a.rp, a.col, a.hash, fc.list[1], (int64_t)s_cnt[1], a.wait, a.color, fn, a.done,
                              sbits);
        if (s_cnt[2])
            color_chunk_items(a.rp, a.col, a.hash, fc.items, (int64_t)s_cnt[2], a.chunk_slot, a.bitmaps,
                              a.chunks_done, a.wait, a.color, fn, a.done, hs, sbits);
        if (!team_sync(tm, &s_gen, &s_ok)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.rounds = r;
}

int32_t color_graph(const GraphView &g, uint64_t seed, int32_t *color, cudaStream_t s) {
    if (g.n == 0) return 0;
    const uint32_t sw = seed_word(seed);
    DBuf<uint32_t> hash(g.n, s);
    DBuf<int32_t> wait(g.n, s);
    // every chunked vertex has more than COLOR_BIG_DEG entries; a frontier holds
    // at most all of their chunks
    const int64_t max_chunked = g.nnz / (COLOR_BIG_DEG + 1) + 1;
    const int64_t icap = g.nnz / COLOR_CHUNK + max_chunked;
    DBuf<int32_t> lists(6 * g.n, s);          // three sides of two vertex tiers
    DBuf<unsigned long long> items(3 * icap, s);
    DBuf<unsigned long long> cnt(10, s);      // [side * 3 + tier], [9] coloured
    DBuf<GridBarrier> bar(1, s);
    DBuf<int64_t> rounds(1, s);
    cnt.zero();
    bar.zero();
    rounds.zero();
    DBuf<int32_t> chunk_slot(g.n, s);
    DBuf<unsigned int> nchunked(1, s);
    nchunked.zero();
    ColorArgs a{};
    a.rp = g.rp;
    a.col = g.col;
    a.hash = hash.p;
    a.n = g.n;
    a.wait = wait.p;
    a.color = color;
    a.lists = lists.p;
    a.items = items.p;
    a.icap = icap;
    a.counts = cnt.p;
    a.done = cnt.p + 9;
    a.chunk_slot = chunk_slot.p;
    a.bar = bar.p;
    a.max_rounds = g.n + 64;   // every round colours at least one vertex
    a.rounds = rounds.p;
    Frontier f0;
    for (int t = 0; t < 2; t++) f0.list[t] = lists.p + (size_t)t * g.n;
    f0.items = items.p;
    for (int t = 0; t < 3; t++) f0.count[t] = cnt.p + t;
    { k_color_init<<<grid_for(g.n * 32, kBlock, 152 * 64), kBlock, 0, s>>>(g.rp, g.col, g.n, sw, hash.p, wait.p, color,
                                                                          f0, chunk_slot.p, nchunked.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    // one colour bitmap and chunk counter per chunked vertex, sized by the
    // count the init kernel took (a bound from nnz alone would be many times
    // larger with a low COLOR_BIG_DEG)
    unsigned int nch = 0;
    CD_CUDA(cudaMemcpyAsync(&nch, nchunked.p, sizeof(nch), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    if ((int64_t)nch > max_chunked)
        raise(CD_ECUDA, "colouring: %u chunked vertices (bound %lld)", nch, (long long)max_chunked);
    DBuf<uint32_t> bitmaps((size_t)nch * COLOR_WORDS, s);
    DBuf<unsigned int> chunks_done(nch, s);
    bitmaps.zero();
    chunks_done.zero();
    a.bitmaps = bitmaps.p;
    a.chunks_done = chunks_done.p;
    // grid: every block resident (the barrier needs it); small graphs take
    // fewer blocks so that concurrent colourings of a batch fit side by side
    int dev = 0, sms = 0, per_sm = 0;
    CD_CUDA(cudaGetDevice(&dev));
    CD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_color_persistent, kBlock, 0));
    if (per_sm < 1) raise(CD_ECUDA, "colouring kernel does not fit on an SM");
    int grid = std::min(sms * per_sm, BARRIER_FAN * BARRIER_SUBS);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (g.n + 2047) / 2048));
    Residency res((const void *)k_color_persistent, grid, 0);   // held until the stream is synchronised below
    void *args[] = {&a};
    CD_CUDA(cudaLaunchCooperativeKernel((const void *)k_color_persistent, dim3(grid), dim3(kBlock), args, 0, s));
    note_launch();
    DBuf<unsigned int> maxc(1, s);
    maxc.zero();
    { k_color_max<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(color, g.n, maxc.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned h(4 * sizeof(unsigned long long));
    CD_CUDA(cudaMemcpyAsync(h.p, cnt.p + 9, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(h.as<unsigned long long>() + 1, maxc.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(h.as<unsigned long long>() + 2, &bar.p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const unsigned long long coloured = h.as<unsigned long long>()[0];
    const unsigned int k = *reinterpret_cast<unsigned int *>(h.as<unsigned long long>() + 1);
    const int err = *reinterpret_cast<int *>(h.as<unsigned long long>() + 2);
    if (err) raise(CD_ETIMEOUT, "a grid barrier of the colouring kernel timed out");
    if ((int64_t)coloured != g.n)
        raise(CD_ECUDA, "colouring stopped with %llu of %lld vertices coloured", coloured, (long long)g.n);
    return (int32_t)k;
}

}  // namespace cd
