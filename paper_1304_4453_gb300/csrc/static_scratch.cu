// cd_modularity_static: modularity of a labelling on a caller-owned device
// CSR without any device allocation.
//
// Some callers cannot allocate device memory when they need an answer: code
// running inside a memory budget that another framework owns completely,
// latency-critical loops that must never reach the allocator (an allocation
// can synchronise the device), or hooks that run while no allocation is
// permitted.  This entry point serves them: its scratch (per-community
// volumes and block partial sums) is one file-scope device array, reserved
// when the library is loaded and kept on every GPU that loads it until the
// process exits.  The array bounds the graph size at STATIC_MAX_VERTICES.
//
// The array's host-side name is only a stand-in: host code obtains its device
// address with cudaGetSymbolAddress, once per device, on the first call made
// with that device current (so that first call belongs before any stream
// capture).  All calls share the array and it keeps the last call's
// contents: every call clears what must start at zero, and calls that overlap
// on the GPU (two streams, or two threads) race on it, so callers serialise
// them.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t STATIC_MAX_VERTICES = int64_t(1) << 20;   // 1,048,576
constexpr int STATIC_BLOCKS = 1024;                          // blocks of the sum of squares
// word layout of the scratch array (64-bit words)
constexpr int64_t OFF_PART = STATIC_MAX_VERTICES;            // 2 words per block
constexpr int64_t OFF_TWOW = OFF_PART + 2 * STATIC_BLOCKS;   // 2 omega(E)
constexpr int64_t OFF_IN2 = OFF_TWOW + 1;                    // sum_C 2 omega(C)
constexpr int64_t OFF_ERR = OFF_IN2 + 1;                     // malformed input seen
constexpr int64_t OFF_RES = OFF_ERR + 1;                     // result (double bits)
constexpr int64_t STATIC_WORDS = OFF_RES + 1;

static __device__ __align__(256) unsigned long long g_static_scratch[STATIC_WORDS];

std::mutex g_mu;
unsigned long long *g_addr[64] = {};

// Device address of the scratch array on the current device.
unsigned long long *scratch_address() {
    int dev = 0;
    CD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) cd::raise(CD_ECUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            cd::raise(CD_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned long long *>(p);
    }
    return g_addr[dev];
}

__global__ void k_static_clear(unsigned long long *s, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 3) s[OFF_TWOW + threadIdx.x] = 0;
}

// One warp per row: 2 omega(C) contributions, vol(u) into its community, 2W.
__global__ void k_static_rows(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                              const int32_t *z, unsigned long long *s) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nnz = rp[n];
    unsigned long long in2 = 0, twoW = 0;
    int bad = 0;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t beg = rp[u], end = rp[u + 1];
        const int32_t cu = z[u];
        // col may be null only when no row has entries (an edgeless graph)
        if (beg < 0 || end < beg || end > nnz || cu < 0 || cu >= n || (!col && end > beg)) { bad = 1; continue; }
        unsigned long long vol = 0, loop = 0, inner = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t v = col[e];
            const unsigned long long we = w ? (unsigned long long)w[e] : 1ull;
            if (v < 0 || v >= n || (w && w[e] <= 0)) { bad = 1; continue; }
            if (v == u) {
                loop += we;
            } else {
                vol += we;
                const int32_t cv = z[v];
                if (cv < 0 || cv >= n) bad = 1;
                else if (cv == cu) inner += we;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            vol += __shfl_xor_sync(0xffffffffu, vol, o);
            loop += __shfl_xor_sync(0xffffffffu, loop, o);
            inner += __shfl_xor_sync(0xffffffffu, inner, o);
        }
        if (lane == 0) {
            const unsigned long long vu = vol + 2 * loop;
            atomicAdd(s + cu, vu);
            twoW += vu;
            in2 += inner + 2 * loop;
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        if (in2) atomicAdd(s + OFF_IN2, in2);
        if (twoW) atomicAdd(s + OFF_TWOW, twoW);
        if (bad) s[OFF_ERR] = 1;
    }
}

__global__ void k_static_squares(unsigned long long *s, int64_t n) {
    __shared__ unsigned long long slo[32], shi[32];
    unsigned __int128 acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned __int128 x = s[i];
        acc += x * x;
    }
    unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)(acc >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const unsigned __int128 t = ((unsigned __int128)hi << 64 | lo) + ((unsigned __int128)h2 << 64 | l2);
        lo = (unsigned long long)t;
        hi = (unsigned long long)(t >> 64);
    }
    if ((threadIdx.x & 31) == 0) { slo[threadIdx.x >> 5] = lo; shi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned __int128 t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += ((unsigned __int128)shi[i] << 64) | slo[i];
        s[OFF_PART + 2 * blockIdx.x] = (unsigned long long)t;
        s[OFF_PART + 2 * blockIdx.x + 1] = (unsigned long long)(t >> 64);
    }
}

// mod = N / D with N = 2W * sum_C 2 omega(C) - sum_C vol(C)^2 and D = (2W)^2.
__global__ void k_static_final(unsigned long long *s, int nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned __int128 sq = 0;
    for (int i = 0; i < nb; i++) sq += ((unsigned __int128)s[OFF_PART + 2 * i + 1] << 64) | s[OFF_PART + 2 * i];
    const __int128 twoW = (__int128)s[OFF_TWOW];
    double r = 0.0;
    if (twoW > 0) {
        const __int128 N = twoW * (__int128)s[OFF_IN2] - (__int128)sq;
        r = cd::i128_to_double(N) / cd::i128_to_double(twoW * twoW);
    }
    s[OFF_RES] = (unsigned long long)__double_as_longlong(r);
}

}  // namespace

extern "C" cd_status cd_modularity_static(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                                          const int32_t *labels, void *stream, double *mod) {
    if (!mod) return CD_EINVAL;
    try {
        if (n < 0 || n > STATIC_MAX_VERTICES)
            cd::raise(CD_EINVAL, "n = %lld is outside [0, %lld], the size of the static scratch", (long long)n,
                      (long long)STATIC_MAX_VERTICES);
        if (!row_ptr || (n > 0 && !labels)) cd::raise(CD_EINVAL, "row_ptr and labels are required");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        unsigned long long *scr = scratch_address();
        const unsigned gv = cd::grid_for(n, cd::kBlock, 152 * 16);
        { k_static_clear<<<gv, cd::kBlock, 0, s>>>(scr, n); cd::note_launch(); }
        { k_static_rows<<<cd::grid_for(n * 32, cd::kBlock, 152 * 32), cd::kBlock, 0, s>>>(n, row_ptr, col, w, labels, scr); cd::note_launch(); }
        const int nb = (int)cd::grid_for(n, cd::kBlock, STATIC_BLOCKS);
        { k_static_squares<<<nb, cd::kBlock, 0, s>>>(scr, n); cd::note_launch(); }
        { k_static_final<<<1, 32, 0, s>>>(scr, nb); cd::note_launch(); }
        CD_LAUNCH_CHECK();
        unsigned long long out[2] = {0, 0};   // error flag, result bits
        CD_CUDA(cudaMemcpyAsync(out, scr + OFF_ERR, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        if (out[0]) cd::raise(CD_EINVAL, "malformed CSR or label out of range [0, n)");
        double r;
        static_assert(sizeof(r) == sizeof(out[1]), "double is 64 bits");
        memcpy(&r, &out[1], sizeof(r));
        *mod = r;
        cd::set_last_error("");
        return CD_OK;
    } catch (const cd::Error &e) {
        cd::set_last_error(e.msg);
        return e.status;
    }
}
