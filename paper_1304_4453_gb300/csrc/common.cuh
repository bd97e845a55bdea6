// Shared declarations of the CUDA library (device helpers, buffers, errors).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "cd.h"

namespace cd {

// ---------------------------------------------------------------------------
// Errors: internal code throws Error; the C ABI catches it and returns the
// status, keeping the message for cd_last_error().
// ---------------------------------------------------------------------------
struct Error {
    cd_status status;
    std::string msg;
};

[[noreturn]] void raise(cd_status s, const char *fmt, ...);
void set_last_error(const std::string &m);

#define CD_CUDA(x)                                                                   \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess)                                                       \
            ::cd::raise(e_ == cudaErrorMemoryAllocation ? CD_ENOMEM : CD_ECUDA,      \
                        "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_),         \
                        __FILE__, __LINE__);                                         \
    } while (0)

#define CD_LAUNCH_CHECK() CD_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// Device memory: stream-ordered allocations from a library-owned pool that
// keeps freed memory reserved, so repeated runs do not return to the driver.
// ---------------------------------------------------------------------------
// Counts kernel launches made by this library (every launch site calls it).
void note_launch();
uint64_t launch_count();

// Bytes of the library's device pool on the current device: in use now, the
// high-water mark of use (reset_high restarts it), and reserved.
void pool_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, bool reset_high);
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
// Test hook: make the k-th next allocation fail with CD_ENOMEM (k <= 0: off).
void set_alloc_failure(int k);

// Persistent kernels (cooperative launches with grid barriers) of this
// library that run at the same time, from any host thread, must fit on the
// device together, or two partly resident grids could each wait for room the
// other holds.  A Residency guard reserves the SM share of one launch
// (blocks / resident blocks per SM) and is held until the kernel has
// finished (the holder synchronises its stream before releasing); it waits
// while the reservations of the other holders leave too little room.
class Residency {
  public:
    Residency(const void *kernel, int blocks, size_t dyn_smem);
    ~Residency();
    Residency(const Residency &) = delete;
    Residency &operator=(const Residency &) = delete;
    int max_blocks() const { return max_blocks_; }   // blocks of this kernel that fit at once
  private:
    int dev_ = 0;
    double share_ = 0;
    int max_blocks_ = 0;
};

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        p = static_cast<T *>(dev_alloc((count ? count : 1) * sizeof(T), st));
    }
    void release() {
        if (p) dev_free(p, s);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    void zero() { CD_CUDA(cudaMemsetAsync(p, 0, (n ? n : 1) * sizeof(T), s)); }
};

// Pinned host staging for small readbacks, recycled per host thread (a
// fresh cudaHostAlloc per readback would cost more than the readback).
struct Pinned {
    void *p = nullptr;
    size_t cap = 0;
    explicit Pinned(size_t bytes);
    ~Pinned();
    Pinned(const Pinned &) = delete;
    Pinned &operator=(const Pinned &) = delete;
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// Graph view used by every kernel: adjacency without self-loops, self-loop
// weights in `self`, vol(u) in `vol`.  Weight kinds: 0 unit (w == nullptr),
// 1 int32, 2 int64.
// ---------------------------------------------------------------------------
enum WKind { W_UNIT = 0, W_I32 = 1, W_I64 = 2 };

struct GraphView {
    int64_t n = 0;
    int64_t nnz = 0;          // adjacency entries (self-loops excluded)
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const void *w = nullptr;
    int wk = W_UNIT;
    const int64_t *self = nullptr;
    const int64_t *vol = nullptr;
    int64_t W = 0;            // omega(E)
    int64_t max_deg = 0;
};

// 2W < 2^31 keeps every gain product below 2^63 and every omega(u, C) below
// 2^31; otherwise the 128-bit path is used.
inline bool needs_big(int64_t W) { return 2 * W >= (int64_t(1) << 31); }

// With a resolution gamma = p/q (Section III-B; p/q reduced) both products of
// the gain are bounded by max(p, q) (2W)^2: the 64-bit path needs that bound
// below 2^63 as well, and no path takes a bound of 2^126 or more
// (gain_fits_128 false: the caller rejects the resolution).
inline bool gain_needs_big(int64_t W, int64_t p, int64_t q) {
    if (needs_big(W)) return true;
    const unsigned __int128 w2 = (unsigned __int128)(2 * W) * (unsigned __int128)(2 * W);
    const unsigned __int128 m = (unsigned __int128)(p > q ? p : q);
    return w2 > 0 && m * w2 >= ((unsigned __int128)1 << 63);
}
inline bool gain_fits_128(int64_t W, int64_t p, int64_t q) {
    const unsigned __int128 w2 = (unsigned __int128)(2 * W) * (unsigned __int128)(2 * W);
    const unsigned __int128 m = (unsigned __int128)(p > q ? p : q);
    return w2 == 0 || m <= (((unsigned __int128)1 << 126) - 1) / w2;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// MurmurHash3 32-bit finaliser (Appleby), a bijection on 32-bit words.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__host__ __device__ __forceinline__ uint32_t seed_word(uint64_t seed) {
    return fmix32(static_cast<uint32_t>(seed) ^ static_cast<uint32_t>(seed >> 32));
}

template <int WK>
__device__ __forceinline__ int64_t edge_weight(const void *w, int64_t e) {
    if constexpr (WK == W_UNIT) return 1;
    else if constexpr (WK == W_I32) return static_cast<const int32_t *>(w)[e];
    else return static_cast<const int64_t *>(w)[e];
}

__device__ __forceinline__ int64_t edge_weight_rt(const void *w, int wk, int64_t e) {
    if (wk == W_UNIT) return 1;
    if (wk == W_I32) return static_cast<const int32_t *>(w)[e];
    return static_cast<const int64_t *>(w)[e];
}

// Correctly rounded (to nearest, ties to even) conversion of a signed 128-bit
// integer to double.
__device__ __forceinline__ double i128_to_double(__int128 x) {
    if (x == 0) return 0.0;
    bool neg = x < 0;
    unsigned __int128 m = neg ? (unsigned __int128)(-(x + 1)) + 1 : (unsigned __int128)x;
    uint64_t hi = (uint64_t)(m >> 64), lo = (uint64_t)m;
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    double r;
    if (msb <= 52) {
        r = (double)lo;  // exact
    } else {
        int sh = msb - 52;
        unsigned __int128 q = m >> sh;
        unsigned __int128 rem = m - (q << sh);
        unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) {
            q += 1;
            if (q >> 53) { q >>= 1; sh += 1; }
        }
        r = ldexp((double)(uint64_t)q, sh);
    }
    return neg ? -r : r;
}

constexpr int kBlock = 256;

// Hubs of the schedule: vertices with more than HUB_RELAX neighbours
// (self-loop not counted).  The colouring ignores edges between two hubs, so
// adjacent hubs may share a colour class and then decide on each other's
// labels as they stood when the class began.
constexpr int64_t HUB_RELAX = 4096;

__device__ __forceinline__ bool relaxed_hub(const int64_t *rp, int32_t v) {
    return rp[v + 1] - rp[v] > HUB_RELAX;
}

inline unsigned grid_for(int64_t items, int per_block, int64_t cap = (int64_t)1 << 30) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g);
}

// ---------------------------------------------------------------------------
// Primitives (primitives.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of `in` (count items) into `out` (count items); the
// total is written to *total_dev if non-null.  In-place allowed.
template <typename Tin>
void exclusive_scan(const Tin *in, int64_t *out, int64_t count, int64_t *total_dev, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs over the 8-bit digits starting
// at each bit position in `digits`.  Sorts in place: keys/vals end holding the
// result (alt buffers are scratch of the same size).
template <typename K, typename V>
void radix_sort_pairs(K *keys, V *vals, K *keys_alt, V *vals_alt, int64_t count,
                      const std::vector<int> &digits, cudaStream_t s);

// Fills out[i] = i.
void iota32(int32_t *out, int64_t n, cudaStream_t s);

// Dense rank of labels: rank_of_label[l] for every used label l in [0, n),
// returns the number of distinct labels (synchronises).  `flags` is scratch
// of n int64.
int64_t dense_rank(const int32_t *labels, int64_t n, int64_t *rank_of_label, cudaStream_t s);
// labels[u] = rank[labels[u]]
void apply_rank(int32_t *labels, const int64_t *rank, int64_t n, cudaStream_t s);
// Compaction in place; returns number of communities.
int64_t compact_labels(int32_t *labels, int64_t n, cudaStream_t s);

// Checks 0 <= labels[u] < n (synchronises); false when out of range.
bool labels_in_range(const int32_t *labels, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Stages
// ---------------------------------------------------------------------------
// Colouring (color.cu).  Returns the number of colours.
int32_t color_graph(const GraphView &g, uint64_t seed, int32_t *color, cudaStream_t s);

// Modularity (modularity.cu).
double modularity(const GraphView &g, const int32_t *labels, cudaStream_t s);

// Owned device graph (coarse levels and API handles).
struct OwnedGraph {
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<int32_t> w32;
    DBuf<int64_t> w64;
    DBuf<int64_t> self;
    DBuf<int64_t> vol;
    GraphView view;
};

// Coarsening (coarsen.cu): one coarse vertex per distinct label.  Computes
// the dense ranks of the labels into rank_of_label (n entries) and builds the
// coarse graph.
// scratch_budget > 0 (the low-memory mode): the sort scratch of one pass
// stays within that many bytes; ranges of coarse rows are coarsened in turn.
void coarsen_graph(const GraphView &g, const int32_t *labels, int64_t *rank_of_label,
                   OwnedGraph &out, cudaStream_t s, int64_t scratch_budget = 0);

}  // namespace cd

// Graph handle of the C ABI.
struct cd_graph {
    cd::OwnedGraph g;
    cudaStream_t stream = nullptr;
    int64_t m = 0;  // undirected loop-free edges of the input
};

namespace cd {
// Optional per-launch CUDA-event timing of the decide kernels.
struct LaunchTimer {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t used = 0;
    void before(cudaStream_t s) {
        if (!on) return;
        if (used == ev.size()) {
            cudaEvent_t a, b;
            CD_CUDA(cudaEventCreate(&a));
            CD_CUDA(cudaEventCreate(&b));
            ev.push_back({a, b});
        }
        CD_CUDA(cudaEventRecord(ev[used].first, s));
    }
    void after(cudaStream_t s) {
        if (!on) return;
        CD_CUDA(cudaEventRecord(ev[used].second, s));
        used++;
    }
    // Sums the recorded durations (the stream must be synchronised).
    double collect_ms() {
        double t = 0;
        for (size_t i = 0; i < used; i++) {
            float ms = 0;
            CD_CUDA(cudaEventElapsedTime(&ms, ev[i].first, ev[i].second));
            t += ms;
        }
        launches += used;
        used = 0;
        return t;
    }
    int64_t launches = 0;
    ~LaunchTimer() {
        for (auto &p : ev) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    }
};
}  // namespace cd
