// Device-wide primitives: exclusive scan, stable LSD radix sort of pairs,
// dense ranking / compaction of labels.
#include "common.cuh"

namespace cd {

// ---------------------------------------------------------------------------
// Block-wide inclusive scan of one int64 per thread (blockDim == kBlock).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t block_inclusive_scan(int64_t x, int64_t *warp_tot, int64_t &block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < kBlock / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kBlock / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    if (warp > 0) x += warp_tot[warp - 1];
    block_total = warp_tot[kBlock / 32 - 1];
    __syncthreads();
    return x;
}

static void scan_geometry(int64_t count, int &nb, int64_t &chunk) {
    int64_t b = (count + 4095) / 4096;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    chunk = (count + b - 1) / b;
    chunk = (chunk + kBlock - 1) / kBlock * kBlock;
    nb = (int)((count + chunk - 1) / chunk);
    if (nb < 1) nb = 1;
}

template <typename Tin>
__global__ void k_scan_reduce(const Tin *in, int64_t count, int64_t chunk, int64_t *partial) {
    __shared__ int64_t wt[kBlock / 32];
    int64_t beg = (int64_t)blockIdx.x * chunk, end = min(count, beg + chunk);
    int64_t acc = 0;
    for (int64_t i = beg + threadIdx.x; i < end; i += kBlock) acc += (int64_t)in[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int i = 0; i < kBlock / 32; i++) t += wt[i];
        partial[blockIdx.x] = t;
    }
}

// Exclusive scan of nb <= 8192 partials by one block; writes the grand total.
__global__ void k_scan_partials(int64_t *partial, int nb, int64_t *total) {
    __shared__ int64_t wt[kBlock / 32];
    int64_t carry = 0;
    for (int base = 0; base < nb; base += kBlock) {
        int i = base + threadIdx.x;
        int64_t x = i < nb ? partial[i] : 0;
        int64_t bt;
        int64_t inc = block_inclusive_scan(x, wt, bt);
        if (i < nb) partial[i] = carry + inc - x;
        carry += bt;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename Tin>
__global__ void k_scan_apply(const Tin *in, int64_t *out, int64_t count, int64_t chunk, const int64_t *partial) {
    __shared__ int64_t wt[kBlock / 32];
    int64_t beg = (int64_t)blockIdx.x * chunk, end = min(count, beg + chunk);
    int64_t carry = partial[blockIdx.x];
    for (int64_t r = beg; r < end; r += kBlock) {
        int64_t i = r + threadIdx.x;
        int64_t x = i < end ? (int64_t)in[i] : 0;
        int64_t bt;
        int64_t inc = block_inclusive_scan(x, wt, bt);
        if (i < end) out[i] = carry + inc - x;
        carry += bt;
    }
}

template <typename Tin>
void exclusive_scan(const Tin *in, int64_t *out, int64_t count, int64_t *total_dev, cudaStream_t s) {
    if (count <= 0) {
        if (total_dev) CD_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
        return;
    }
    int nb;
    int64_t chunk;
    scan_geometry(count, nb, chunk);
    DBuf<int64_t> partial(nb, s);
    { k_scan_reduce<Tin><<<nb, kBlock, 0, s>>>(in, count, chunk, partial.p); ::cd::note_launch(); }
    { k_scan_partials<<<1, kBlock, 0, s>>>(partial.p, nb, total_dev); ::cd::note_launch(); }
    { k_scan_apply<Tin><<<nb, kBlock, 0, s>>>(in, out, count, chunk, partial.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

template void exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<uint32_t>(const uint32_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<uint8_t>(const uint8_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<unsigned long long>(const unsigned long long *, int64_t *, int64_t, int64_t *,
                                                  cudaStream_t);

// ---------------------------------------------------------------------------
// Radix sort: per block digit histograms -> global offsets (digit-major scan)
// -> stable scatter.  A block owns a contiguous chunk and walks it in rounds
// of kBlock elements; inside a round, ranks come from warp match masks and a
// per-digit prefix over the warps, which keeps equal digits in input order.
// ---------------------------------------------------------------------------
static void sort_geometry(int64_t count, int &nb, int64_t &chunk) {
    int64_t b = (count + 8191) / 8192;
    if (b > 2048) b = 2048;
    if (b < 1) b = 1;
    chunk = (count + b - 1) / b;
    chunk = (chunk + kBlock - 1) / kBlock * kBlock;
    nb = (int)((count + chunk - 1) / chunk);
    if (nb < 1) nb = 1;
}

template <typename K>
__global__ void k_rs_hist(const K *keys, int64_t count, int64_t chunk, int shift, uint32_t *hist, int nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t beg = (int64_t)blockIdx.x * chunk, end = min(count, beg + chunk);
    for (int64_t i = beg + threadIdx.x; i < end; i += kBlock)
        atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <typename K, typename V>
__global__ void k_rs_scatter(const K *kin, const V *vin, K *kout, V *vout, int64_t count, int64_t chunk,
                             int shift, const int64_t *offs, int nb) {
    __shared__ int64_t base[256];
    __shared__ uint32_t wcnt[kBlock / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * nb + blockIdx.x];
#pragma unroll
    for (int j = 0; j < kBlock / 32; j++) wcnt[j][tid] = 0;
    __syncthreads();
    int64_t beg = (int64_t)blockIdx.x * chunk, end = min(count, beg + chunk);
    for (int64_t r = beg; r < end; r += kBlock) {
        int64_t i = r + tid;
        bool valid = i < end;
        K k = valid ? kin[i] : K(0);
        V v = valid ? vin[i] : V(0);
        uint32_t d = valid ? ((uint32_t)(k >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < kBlock / 32; j++) {
            uint32_t c = wcnt[j][tid];
            wcnt[j][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base[tid] += run;
#pragma unroll
        for (int j = 0; j < kBlock / 32; j++) wcnt[j][tid] = 0;
        __syncthreads();
    }
}

template <typename K, typename V>
void radix_sort_pairs(K *keys, V *vals, K *keys_alt, V *vals_alt, int64_t count,
                      const std::vector<int> &digits, cudaStream_t s) {
    if (count <= 1 || digits.empty()) return;
    int nb;
    int64_t chunk;
    sort_geometry(count, nb, chunk);
    DBuf<uint32_t> hist((size_t)256 * nb, s);
    DBuf<int64_t> offs((size_t)256 * nb, s);
    K *ka = keys, *kb = keys_alt;
    V *va = vals, *vb = vals_alt;
    for (int shift : digits) {
        { k_rs_hist<K><<<nb, kBlock, 0, s>>>(ka, count, chunk, shift, hist.p, nb); ::cd::note_launch(); }
        exclusive_scan<uint32_t>(hist.p, offs.p, (int64_t)256 * nb, nullptr, s);
        { k_rs_scatter<K, V><<<nb, kBlock, 0, s>>>(ka, va, kb, vb, count, chunk, shift, offs.p, nb); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CD_CUDA(cudaMemcpyAsync(keys, ka, count * sizeof(K), cudaMemcpyDeviceToDevice, s));
        CD_CUDA(cudaMemcpyAsync(vals, va, count * sizeof(V), cudaMemcpyDeviceToDevice, s));
    }
}

template void radix_sort_pairs<uint32_t, int32_t>(uint32_t *, int32_t *, uint32_t *, int32_t *, int64_t,
                                                   const std::vector<int> &, cudaStream_t);
template void radix_sort_pairs<uint64_t, int32_t>(uint64_t *, int32_t *, uint64_t *, int32_t *, int64_t,
                                                   const std::vector<int> &, cudaStream_t);
template void radix_sort_pairs<uint64_t, int64_t>(uint64_t *, int64_t *, uint64_t *, int64_t *, int64_t,
                                                   const std::vector<int> &, cudaStream_t);

// ---------------------------------------------------------------------------
// Labels
// ---------------------------------------------------------------------------
__global__ void k_iota32(int32_t *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

void iota32(int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    { k_iota32<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(out, n); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

__global__ void k_mark_used(const int32_t *labels, int64_t n, int64_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flags[labels[i]] = 1;
}

int64_t dense_rank(const int32_t *labels, int64_t n, int64_t *rank_of_label, cudaStream_t s) {
    if (n <= 0) return 0;
    CD_CUDA(cudaMemsetAsync(rank_of_label, 0, n * sizeof(int64_t), s));
    { k_mark_used<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(labels, n, rank_of_label); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    DBuf<int64_t> total(1, s);
    exclusive_scan<int64_t>(rank_of_label, rank_of_label, n, total.p, s);
    Pinned h(sizeof(int64_t));
    CD_CUDA(cudaMemcpyAsync(h.p, total.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return *h.as<int64_t>();
}

__global__ void k_apply_rank(int32_t *labels, const int64_t *rank, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        labels[i] = (int32_t)rank[labels[i]];
}

void apply_rank(int32_t *labels, const int64_t *rank, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    { k_apply_rank<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(labels, rank, n); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

int64_t compact_labels(int32_t *labels, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    DBuf<int64_t> rank(n, s);
    int64_t k = dense_rank(labels, n, rank.p, s);
    apply_rank(labels, rank.p, n, s);
    return k;
}

__global__ void k_range(const int32_t *labels, int64_t n, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (labels[i] < 0 || labels[i] >= n) *bad = 1;
}

bool labels_in_range(const int32_t *labels, int64_t n, cudaStream_t s) {
    if (n <= 0) return true;
    DBuf<int> bad(1, s);
    bad.zero();
    { k_range<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(labels, n, bad.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned h(sizeof(int));
    CD_CUDA(cudaMemcpyAsync(h.p, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return *h.as<int>() == 0;
}

}  // namespace cd
