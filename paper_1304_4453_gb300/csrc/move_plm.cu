// PLM / PLMR decide kernels (Algorithm 2) and the volume update of moves.
#include "move_dispatch.cuh"

namespace cd {

__global__ void k_apply_moves(const int32_t *mv_u, const int32_t *mv_c, const unsigned long long *nmv,
                              const int32_t *zeta, const int64_t *vol, int64_t *volc) {
    const int64_t cnt = (int64_t)*nmv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = mv_u[i];
        const int64_t vu = vol[u];
        atomicAdd(reinterpret_cast<unsigned long long *>(volc + mv_c[i]), (unsigned long long)(-vu));
        atomicAdd(reinterpret_cast<unsigned long long *>(volc + zeta[u]), (unsigned long long)vu);
    }
}

// ---------------------------------------------------------------------------
// Sequential re-check of one class's wanted moves (sweeps >= the re-check
// sweep).  The candidates are sorted by vertex id (bitonic sort in shared
// memory, or a block-wide LSD radix sort in global scratch for large lists);
// then warp 0 walks them in windows of 32: lane k recomputes its gain with the
// volumes of its source and target as updated by every move accepted before
// it, and every later lane of the window adjusts its copies of the volumes
// it shares with an accepted move.  Accepted moves update zeta and the
// community volumes before the next window loads its volumes.
// ---------------------------------------------------------------------------
constexpr int RC_THREADS = 1024;
constexpr int RC_SMALL = 4096;

__device__ void rc_radix_pass(const uint64_t *in, uint64_t *out, int64_t m, int shift, unsigned char *smem) {
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(smem);                     // [32][256]
    int64_t *base = reinterpret_cast<int64_t *>(smem + 32 * 256 * 4);       // [256]
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + 32 * 256 * 4 + 256 * 8);  // [256]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 256) hist[tid] = 0;
    for (int j = tid; j < 32 * 256; j += RC_THREADS) wcnt[j] = 0;
    __syncthreads();
    for (int64_t i = tid; i < m; i += RC_THREADS) atomicAdd(&hist[(uint32_t)(in[i] >> shift) & 255u], 1u);
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int d = 0; d < 256; d++) { base[d] = run; run += hist[d]; }
    }
    __syncthreads();
    for (int64_t r = 0; r < m; r += RC_THREADS) {
        const int64_t i = r + tid;
        const bool valid = i < m;
        const uint64_t k = valid ? in[i] : 0;
        const uint32_t d = valid ? ((uint32_t)(k >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp * 256 + d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        if (tid < 256)
            for (int j = 0; j < 32; j++) {
                uint32_t c = wcnt[j * 256 + tid];
                wcnt[j * 256 + tid] = run;
                run += c;
            }
        __syncthreads();
        if (valid) out[base[d] + wcnt[warp * 256 + d] + rank] = k;
        __syncthreads();
        if (tid < 256) {
            base[tid] += run;
            for (int j = 0; j < 32; j++) wcnt[j * 256 + tid] = 0;
        }
        __syncthreads();
    }
}

template <bool BIG>
__global__ void __launch_bounds__(RC_THREADS) k_recheck(RecheckArgs a) {
    __shared__ __align__(16) unsigned char smem[36 * 1024];
    const int64_t m = (int64_t)*a.ncand;
    if (m == 0) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t *keys;
    if (m <= RC_SMALL) {
        uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
        int P = 1;
        while (P < m) P <<= 1;
        for (int i = tid; i < P; i += RC_THREADS)
            sk[i] = i < m ? (((uint64_t)(uint32_t)a.cu[i] << 32) | (uint32_t)i) : ~0ull;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < P; i += RC_THREADS) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const bool up = (i & k) == 0;
                        const uint64_t x = sk[i], y = sk[ixj];
                        if ((x > y) == up) { sk[i] = y; sk[ixj] = x; }
                    }
                }
                __syncthreads();
            }
        keys = sk;
    } else {
        for (int64_t i = tid; i < m; i += RC_THREADS)
            a.tmp_a[i] = ((uint64_t)(uint32_t)a.cu[i] << 32) | (uint32_t)i;
        __syncthreads();
        uint64_t *src = a.tmp_a, *dst = a.tmp_b;
        for (int shift = 32; shift < 32 + a.ubits; shift += 8) {
            rc_radix_pass(src, dst, m, shift, smem);
            uint64_t *t = src; src = dst; dst = t;
        }
        __threadfence_block();
        __syncthreads();
        keys = src;
    }
    if (tid >= 32) return;
    unsigned long long moved = 0;
    for (int64_t w0 = 0; w0 < m; w0 += 32) {
        const int64_t i = w0 + lane;
        const bool valid = i < m;
        const uint32_t ci = valid ? (uint32_t)(keys[i] & 0xffffffffull) : 0u;
        const int32_t u = valid ? a.cu[ci] : 0;
        const int32_t C = valid ? a.cc[ci] : -1;
        const int32_t D = valid ? a.cd[ci] : -2;
        const int64_t vu = valid ? a.vol[u] : 0;
        const int64_t wD = valid ? a.cwd[ci] : 0, wC = valid ? a.cwc[ci] : 0;
        int64_t volC = valid ? __ldcg(a.volc + C) : 0;
        int64_t volD = valid ? __ldcg(a.volc + D) : 0;
        bool mine = false;
        const int cnt = (m - w0) < 32 ? (int)(m - w0) : 32;
        for (int k = 0; k < cnt; k++) {
            int acc = 0;
            if (lane == k) acc = plm_gain<BIG>(a.twoW, wD, wC, vu, volD, volC) > 0;
            acc = __shfl_sync(0xffffffffu, acc, k);
            if (acc) {
                const int32_t Ck = __shfl_sync(0xffffffffu, C, k), Dk = __shfl_sync(0xffffffffu, D, k);
                const int64_t vk = __shfl_sync(0xffffffffu, vu, k);
                if (lane == k) {
                    mine = true;
                } else if (lane > k) {
                    if (C == Ck) volC -= vk; else if (C == Dk) volC += vk;
                    if (D == Ck) volD -= vk; else if (D == Dk) volD += vk;
                }
            }
        }
        if (valid && mine) {
            a.zeta[u] = D;
            atomicAdd(reinterpret_cast<unsigned long long *>(a.volc + C), (unsigned long long)(-vu));
            atomicAdd(reinterpret_cast<unsigned long long *>(a.volc + D), (unsigned long long)vu);
        }
        moved += __popc(__ballot_sync(0xffffffffu, valid && mine));
        __syncwarp();
    }
    if (lane == 0 && moved) atomicAdd(&a.cnt->moved, moved);
}

void recheck_class(bool big, const RecheckArgs &a, cudaStream_t s) {
    if (big) { k_recheck<true><<<1, RC_THREADS, 0, s>>>(a); ::cd::note_launch(); }
    else { k_recheck<false><<<1, RC_THREADS, 0, s>>>(a); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

template <>
void decide_class<false>(int wk, bool big, const SweepCtx &c, const ClassBins &cb, cudaStream_t s, LaunchTimer &t) {
    if (!big) {
        if (wk == W_UNIT) decide_class_t<W_UNIT, false, false>(c, cb, s, t);
        else if (wk == W_I32) decide_class_t<W_I32, false, false>(c, cb, s, t);
        else raise(CD_ECUDA, "int64 weights need the 128-bit gain path");
    } else {
        if (wk == W_UNIT) decide_class_t<W_UNIT, true, false>(c, cb, s, t);
        else if (wk == W_I32) decide_class_t<W_I32, true, false>(c, cb, s, t);
        else decide_class_t<W_I64, true, false>(c, cb, s, t);
    }
}

}  // namespace cd
