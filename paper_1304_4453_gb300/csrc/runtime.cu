// Runtime support: error reporting, the device memory pool, pinned staging,
// and the residency budget of concurrent persistent kernels.
#include <atomic>
#include <condition_variable>
#include <mutex>

#include "common.cuh"

namespace cd {

static thread_local std::string t_last_error;

void set_last_error(const std::string &m) { t_last_error = m; }
const std::string &last_error() { return t_last_error; }

[[noreturn]] void raise(cd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error{s, std::string(buf)};
}

// One pool per device, created on first use.  Its release threshold is the
// maximum, so memory freed at the end of a run stays reserved for the next.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};
static std::atomic<int> g_fail_countdown{0};
static std::atomic<uint64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_alloc_failure(int k) { g_fail_countdown.store(k > 0 ? k : 0); }

static cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    CD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) raise(CD_ECUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        CD_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t thr = ~0ull;
        CD_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
    int k = g_fail_countdown.load();
    if (k > 0) {
        if (g_fail_countdown.fetch_sub(1) == 1)
            raise(CD_ENOMEM, "injected allocation failure (%zu bytes)", bytes);
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool_for_current_device(), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        raise(e == cudaErrorMemoryAllocation ? CD_ENOMEM : CD_ECUDA,
              "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return p;
}

void pool_stats(uint64_t *used, uint64_t *used_high, uint64_t *reserved, bool reset_high) {
    cudaMemPool_t p = pool_for_current_device();
    uint64_t v = 0;
    if (used) { CD_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &v)); *used = v; }
    if (used_high) { CD_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemHigh, &v)); *used_high = v; }
    if (reserved) { CD_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &v)); *reserved = v; }
    if (reset_high) {
        uint64_t zero = 0;
        CD_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrUsedMemHigh, &zero));
    }
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);  // never throws (destructors)
}

static std::mutex g_res_mu;
static std::condition_variable g_res_cv;
static double g_res_used[64] = {};

Residency::Residency(const void *kernel, int blocks, size_t dyn_smem) {
    int sms = 0, per_sm = 0;
    CD_CUDA(cudaGetDevice(&dev_));
    if (dev_ < 0 || dev_ >= 64) raise(CD_ECUDA, "device ordinal %d out of range", dev_);
    CD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_));
    CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, dyn_smem));
    if (per_sm < 1) raise(CD_ECUDA, "persistent kernel does not fit on an SM");
    max_blocks_ = sms * per_sm;
    if (blocks > max_blocks_) raise(CD_ECUDA, "persistent grid of %d blocks exceeds %d resident blocks", blocks,
                                    max_blocks_);
    share_ = (double)blocks / per_sm;
    std::unique_lock<std::mutex> lk(g_res_mu);
    // a launch that needs the whole device still proceeds when it is alone
    g_res_cv.wait(lk, [&]() { return g_res_used[dev_] == 0.0 || g_res_used[dev_] + share_ <= sms + 1e-9; });
    g_res_used[dev_] += share_;
}

Residency::~Residency() {
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        g_res_used[dev_] -= share_;
        if (g_res_used[dev_] < 1e-9) g_res_used[dev_] = 0.0;
    }
    g_res_cv.notify_all();
}

namespace {
struct PinnedCache {
    std::vector<std::pair<size_t, void *>> blocks;   // (capacity, pointer), free
    ~PinnedCache() {
        for (auto &b : blocks) cudaFreeHost(b.second);
    }
};
thread_local PinnedCache t_pinned;
constexpr size_t PINNED_KEEP = 16;   // free blocks kept per thread
}  // namespace

Pinned::Pinned(size_t bytes) {
    auto &fl = t_pinned.blocks;
    int best = -1;
    for (int i = 0; i < (int)fl.size(); i++)
        if (fl[i].first >= bytes && (best < 0 || fl[i].first < fl[best].first)) best = i;
    if (best >= 0) {
        cap = fl[best].first;
        p = fl[best].second;
        fl.erase(fl.begin() + best);
        return;
    }
    cap = 256;
    while (cap < bytes) cap <<= 1;
    CD_CUDA(cudaHostAlloc(&p, cap, cudaHostAllocDefault));
}

Pinned::~Pinned() {
    if (!p) return;
    auto &fl = t_pinned.blocks;
    if (fl.size() >= PINNED_KEEP) {
        int small = 0;
        for (int i = 1; i < (int)fl.size(); i++)
            if (fl[i].first < fl[small].first) small = i;
        cudaFreeHost(fl[small].second);
        fl.erase(fl.begin() + small);
    }
    fl.push_back({cap, p});
}

}  // namespace cd
