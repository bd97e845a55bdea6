// Modularity, Eq. (1), evaluated exactly:
//   mod = N / D,  N = 2W * sum_C 2 omega(C) - sum_C vol(C)^2,  D = 4 W^2,
// with sum_C 2 omega(C) = sum over adjacency entries inside a community of
// their weight + 2 * sum of self-loops.  N and D are exact 128-bit integers,
// each rounded once to double, then one IEEE division.
#include "common.cuh"

namespace cd {

template <int WK>
__global__ void k_mod_rows(GraphView g, const int32_t *__restrict__ z, unsigned long long *volc,
                           unsigned long long *in2) {
    __shared__ int64_t sh[kBlock / 32];
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t acc = 0;
    for (int64_t u = warp; u < g.n; u += nwarps) {
        const int32_t cu = z[u];
        const int64_t beg = g.rp[u], end = g.rp[u + 1];
        for (int64_t e = beg + lane; e < end; e += 32)
            if (z[g.col[e]] == cu) acc += edge_weight<WK>(g.w, e);
        if (lane == 0) {
            acc += 2 * g.self[u];
            atomicAdd(volc + cu, (unsigned long long)g.vol[u]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int i = 0; i < kBlock / 32; i++) t += sh[i];
        atomicAdd(in2, (unsigned long long)t);
    }
}

__global__ void k_mod_sq(const unsigned long long *volc, int64_t n, unsigned long long *part) {
    __shared__ unsigned long long slo[kBlock / 32], shi[kBlock / 32];
    unsigned __int128 acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned __int128 x = volc[i];
        acc += x * x;
    }
    unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)(acc >> 64);
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        unsigned __int128 s = ((unsigned __int128)hi << 64 | lo) + ((unsigned __int128)h2 << 64 | l2);
        lo = (unsigned long long)s;
        hi = (unsigned long long)(s >> 64);
    }
    if ((threadIdx.x & 31) == 0) { slo[threadIdx.x >> 5] = lo; shi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned __int128 t = 0;
        for (int i = 0; i < kBlock / 32; i++) t += ((unsigned __int128)shi[i] << 64) | slo[i];
        part[2 * blockIdx.x] = (unsigned long long)t;
        part[2 * blockIdx.x + 1] = (unsigned long long)(t >> 64);
    }
}

__global__ void k_mod_final(const unsigned long long *part, int nb, const unsigned long long *in2, int64_t W,
                            double *out) {
    if (threadIdx.x != 0) return;
    unsigned __int128 sq = 0;
    for (int i = 0; i < nb; i++) sq += ((unsigned __int128)part[2 * i + 1] << 64) | part[2 * i];
    __int128 N = (__int128)(2 * W) * (__int128)(int64_t)*in2 - (__int128)sq;
    __int128 D = (__int128)4 * W * W;
    *out = i128_to_double(N) / i128_to_double(D);
}

double modularity(const GraphView &g, const int32_t *labels, cudaStream_t s) {
    if (g.W == 0 || g.n == 0) return 0.0;
    DBuf<unsigned long long> volc(g.n, s), in2(1, s);
    volc.zero();
    in2.zero();
    const unsigned gw = grid_for(g.n * 32, kBlock, 152 * 64);
    if (g.wk == W_UNIT) { k_mod_rows<W_UNIT><<<gw, kBlock, 0, s>>>(g, labels, volc.p, in2.p); ::cd::note_launch(); }
    else if (g.wk == W_I32) { k_mod_rows<W_I32><<<gw, kBlock, 0, s>>>(g, labels, volc.p, in2.p); ::cd::note_launch(); }
    else { k_mod_rows<W_I64><<<gw, kBlock, 0, s>>>(g, labels, volc.p, in2.p); ::cd::note_launch(); }
    const int nb = (int)grid_for(g.n, kBlock, 152 * 8);
    DBuf<unsigned long long> part(2 * nb, s);
    { k_mod_sq<<<nb, kBlock, 0, s>>>(volc.p, g.n, part.p); ::cd::note_launch(); }
    DBuf<double> res(1, s);
    { k_mod_final<<<1, 32, 0, s>>>(part.p, nb, in2.p, g.W, res.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned h(sizeof(double));
    CD_CUDA(cudaMemcpyAsync(h.p, res.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    return *h.as<double>();
}

}  // namespace cd
