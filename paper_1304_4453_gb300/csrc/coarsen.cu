// coarsen (Section III-B): communities become coarse vertices numbered by the
// dense rank of their label; weights between communities are summed into
// coarse edges; weight inside a community (its internal edges once, plus the
// self-loops of its members) becomes the coarse self-loop.
//
// Steps: dense rank of the labels (prefix sum over used-label flags), one
// pass per row that counts inter-community entries and accumulates the
// intra-community weight per coarse vertex, a second pass that emits
// (pi(u) << 32 | pi(v), w) for inter-community entries, a stable LSD radix
// sort of those keys, and a segmented reduction of equal keys into the
// coarse CSR (rows sorted by column because the keys are).
#include "common.cuh"
#include "graph.cuh"

namespace cd {

template <int WK>
__global__ void k_coarse_count(GraphView g, const int32_t *__restrict__ zeta, const int64_t *__restrict__ rank,
                               int64_t *inter, unsigned long long *intra2) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < g.n; u += nwarps) {
        const int64_t cu = rank[zeta[u]];
        const int64_t beg = g.rp[u], end = g.rp[u + 1];
        int64_t cnt = 0, in = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            if (rank[zeta[g.col[e]]] == cu) in += edge_weight<WK>(g.w, e);
            else cnt++;
        }
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            in += __shfl_xor_sync(0xffffffffu, in, o);
        }
        if (lane == 0) {
            inter[u] = cnt;
            // sum over members of (intra entries + 2 * loop) = 2 * coarse loop
            atomicAdd(intra2 + cu, (unsigned long long)(in + 2 * g.self[u]));
        }
    }
}

// Emits the inter-community entries of the rows whose coarse vertex lies in
// [c_lo, c_hi) (every row when the range covers all coarse vertices).
template <int WK>
__global__ void k_coarse_emit(GraphView g, const int32_t *__restrict__ zeta, const int64_t *__restrict__ rank,
                              const int64_t *__restrict__ pos, uint64_t *keys, int64_t *wv, int64_t c_lo,
                              int64_t c_hi) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < g.n; u += nwarps) {
        const uint64_t cu = (uint64_t)rank[zeta[u]];
        if ((int64_t)cu < c_lo || (int64_t)cu >= c_hi) continue;
        const int64_t beg = g.rp[u], end = g.rp[u + 1];
        int64_t out = pos[u];
        for (int64_t e0 = beg; e0 < end; e0 += 32) {
            const int64_t e = e0 + lane;
            uint64_t cv = 0;
            bool inter = false;
            if (e < end) {
                cv = (uint64_t)rank[zeta[g.col[e]]];
                inter = cv != cu;
            }
            unsigned b = __ballot_sync(0xffffffffu, inter);
            if (inter) {
                const int64_t o = out + __popc(b & ((1u << lane) - 1u));
                keys[o] = (cu << 32) | cv;
                wv[o] = edge_weight<WK>(g.w, e);
            }
            out += __popc(b);
        }
    }
}

// Heads of equal-key runs.
__global__ void k_heads(const uint64_t *keys, int64_t cnt, int32_t *head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Segmented sum of the weights of each run (warp segmented scan, one atomic
// per run per warp), coarse column at the run head, row entry counts.
__global__ void k_reduce_runs(const uint64_t *keys, const int64_t *wv, const int64_t *uidx_excl, int64_t cnt,
                              int32_t *ocol, unsigned long long *ow, unsigned long long *rowcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wb = warp * 32; wb < cnt; wb += nwarps * 32) {
        const int64_t i = wb + lane;
        const bool ok = i < cnt;
        const uint64_t k = ok ? keys[i] : ~0ull;
        const int64_t id = ok ? uidx_excl[i] + ((i == 0 || keys[i] != keys[i - 1]) ? 1 : 0) - 1 : -1;
        int64_t v = ok ? wv[i] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            int64_t idy = __shfl_up_sync(0xffffffffu, id, o);
            if (lane >= o && idy == id) v += y;
        }
        const int64_t idn = __shfl_down_sync(0xffffffffu, id, 1);
        const bool last = lane == 31 || idn != id;
        if (ok && last) atomicAdd(ow + id, (unsigned long long)v);
        if (ok && (i == 0 || keys[i] != keys[i - 1])) {
            ocol[id] = (int32_t)(k & 0xffffffffull);
            atomicAdd(rowcnt + (k >> 32), 1ull);
        }
    }
}

// Inter-community entries per coarse vertex, and per fine row only for the
// rows of one range of coarse vertices (streaming coarsening).
__global__ void k_coarse_row_sums(const int32_t *zeta, const int64_t *rank, const int64_t *inter, int64_t n,
                                  unsigned long long *csum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (inter[i]) atomicAdd(csum + rank[zeta[i]], (unsigned long long)inter[i]);
}

__global__ void k_inter_in_range(const int32_t *zeta, const int64_t *rank, const int64_t *inter, int64_t n,
                                 int64_t c_lo, int64_t c_hi, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = rank[zeta[i]];
        out[i] = (c >= c_lo && c < c_hi) ? inter[i] : 0;
    }
}

__global__ void k_finish_self(const unsigned long long *intra2, int64_t n, int64_t *self) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        self[i] = (int64_t)(intra2[i] / 2);
}

__global__ void k_to_i32(const unsigned long long *in, int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

static int bits_for(int64_t x) {   // bits to represent values < x
    int b = 1;
    while (((int64_t)1 << b) < x) b++;
    return b;
}

// Sort, run detection and segmented sum of T emitted entries: the coarse
// columns and summed weights of their runs are appended to col_out / w_out
// (device buffers of the run count), and rowcnt[c] counts the runs of row c.
static void reduce_chunk(DBuf<uint64_t> &keys, DBuf<int64_t> &wv, int64_t T, int64_t nc,
                         std::vector<DBuf<int32_t>> &col_out, std::vector<DBuf<unsigned long long>> &w_out,
                         unsigned long long *rowcnt, cudaStream_t s) {
    {
        DBuf<uint64_t> keys2(T, s);
        DBuf<int64_t> wv2(T, s);
        std::vector<int> digits;
        const int b = bits_for(nc);
        for (int d = 0; d < b; d += 8) digits.push_back(d);
        for (int d = 0; d < b; d += 8) digits.push_back(32 + d);
        radix_sort_pairs<uint64_t, int64_t>(keys.p, wv.p, keys2.p, wv2.p, T, digits, s);
    }
    DBuf<int32_t> head(T, s);
    DBuf<int64_t> uidx(T, s), tot(1, s);
    { k_heads<<<grid_for(T, kBlock, 152 * 32), kBlock, 0, s>>>(keys.p, T, head.p); ::cd::note_launch(); }
    exclusive_scan<int32_t>(head.p, uidx.p, T, tot.p, s);
    Pinned h(sizeof(int64_t));
    CD_CUDA(cudaMemcpyAsync(h.p, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const int64_t U = *h.as<int64_t>();
    col_out.emplace_back(U, s);
    w_out.emplace_back(U, s);
    w_out.back().zero();
    { k_reduce_runs<<<grid_for(T, kBlock, 152 * 32), kBlock, 0, s>>>(keys.p, wv.p, uidx.p, T, col_out.back().p,
                                                                   w_out.back().p, rowcnt); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

template <int WK>
static void emit(const GraphView &g, const int32_t *zeta, const int64_t *rank, const int64_t *pos, uint64_t *keys,
                 int64_t *wv, int64_t c_lo, int64_t c_hi, unsigned gw, cudaStream_t s) {
    k_coarse_emit<WK><<<gw, kBlock, 0, s>>>(g, zeta, rank, pos, keys, wv, c_lo, c_hi);
    ::cd::note_launch();
    CD_LAUNCH_CHECK();
}

// Bytes of coarsening scratch per emitted entry: keys and weights with their
// sort buffers (32), run heads (4), run ranks (8) and the summed weight (8).
constexpr int64_t COARSEN_BYTES_PER_ENTRY = 52;

void coarsen_graph(const GraphView &g, const int32_t *zeta, int64_t *rank, OwnedGraph &out, cudaStream_t s,
                   int64_t scratch_budget) {
    const int64_t nc = dense_rank(zeta, g.n, rank, s);
    const bool big = needs_big(g.W);
    DBuf<int64_t> inter(g.n + 1, s), pos(g.n + 1, s);
    DBuf<unsigned long long> intra2(nc, s);
    intra2.zero();
    CD_CUDA(cudaMemsetAsync(inter.p + g.n, 0, sizeof(int64_t), s));
    const unsigned gw = grid_for(g.n * 32, kBlock, 152 * 64);
    if (g.n) {
        if (g.wk == W_UNIT) { k_coarse_count<W_UNIT><<<gw, kBlock, 0, s>>>(g, zeta, rank, inter.p, intra2.p); ::cd::note_launch(); }
        else if (g.wk == W_I32) { k_coarse_count<W_I32><<<gw, kBlock, 0, s>>>(g, zeta, rank, inter.p, intra2.p); ::cd::note_launch(); }
        else { k_coarse_count<W_I64><<<gw, kBlock, 0, s>>>(g, zeta, rank, inter.p, intra2.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
    }
    DBuf<int64_t> tot(1, s);
    exclusive_scan<int64_t>(inter.p, pos.p, g.n + 1, tot.p, s);
    Pinned h(sizeof(int64_t));
    CD_CUDA(cudaMemcpyAsync(h.p, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const int64_t T = *h.as<int64_t>();

    // Ranges of coarse rows, each emitting at most `cap` entries (a single row
    // above the cap forms its own range): one range unless a scratch budget
    // is set and the whole emission would exceed it (streaming coarsening,
    // the low-memory mode).  Rows are never split, so every range sorts and
    // reduces complete rows and the result does not depend on the ranges.
    std::vector<int64_t> cut{0, nc};
    if (scratch_budget > 0 && T * COARSEN_BYTES_PER_ENTRY > scratch_budget && nc > 1) {
        const int64_t cap = std::max<int64_t>(1, scratch_budget / COARSEN_BYTES_PER_ENTRY);
        DBuf<unsigned long long> csum(nc, s);
        csum.zero();
        { k_coarse_row_sums<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(zeta, rank, inter.p, g.n, csum.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        std::vector<unsigned long long> hs(nc);
        CD_CUDA(cudaMemcpyAsync(hs.data(), csum.p, nc * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        cut.assign(1, 0);
        int64_t run = 0;
        for (int64_t c = 0; c < nc; c++) {
            if (run > 0 && run + (int64_t)hs[c] > cap) {
                cut.push_back(c);
                run = 0;
            }
            run += (int64_t)hs[c];
        }
        cut.push_back(nc);
    }
    std::vector<DBuf<int32_t>> cols;
    std::vector<DBuf<unsigned long long>> ws;
    DBuf<unsigned long long> rowcnt(nc + 1, s);
    rowcnt.zero();
    for (size_t r = 0; r + 1 < cut.size(); r++) {
        const int64_t c_lo = cut[r], c_hi = cut[r + 1];
        int64_t Tr = T;
        const int64_t *pr = pos.p;
        DBuf<int64_t> inter_r, pos_r;
        if (cut.size() > 2) {
            inter_r.alloc(g.n + 1, s);
            pos_r.alloc(g.n + 1, s);
            CD_CUDA(cudaMemsetAsync(inter_r.p + g.n, 0, sizeof(int64_t), s));
            if (g.n) { k_inter_in_range<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(zeta, rank, inter.p, g.n, c_lo, c_hi, inter_r.p); ::cd::note_launch(); }
            CD_LAUNCH_CHECK();
            exclusive_scan<int64_t>(inter_r.p, pos_r.p, g.n + 1, tot.p, s);
            CD_CUDA(cudaMemcpyAsync(h.p, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CD_CUDA(cudaStreamSynchronize(s));
            Tr = *h.as<int64_t>();
            pr = pos_r.p;
        }
        if (Tr == 0) continue;
        DBuf<uint64_t> keys(Tr, s);
        DBuf<int64_t> wv(Tr, s);
        if (g.wk == W_UNIT) emit<W_UNIT>(g, zeta, rank, pr, keys.p, wv.p, c_lo, c_hi, gw, s);
        else if (g.wk == W_I32) emit<W_I32>(g, zeta, rank, pr, keys.p, wv.p, c_lo, c_hi, gw, s);
        else emit<W_I64>(g, zeta, rank, pr, keys.p, wv.p, c_lo, c_hi, gw, s);
        reduce_chunk(keys, wv, Tr, nc, cols, ws, rowcnt.p, s);
    }
    int64_t U = 0;
    for (const auto &c : cols) U += (int64_t)c.n;
    out = OwnedGraph();
    GraphView &v = out.view;
    v.n = nc;
    v.nnz = U;
    v.wk = big ? W_I64 : W_I32;
    out.rp.alloc(nc + 1, s);
    exclusive_scan<unsigned long long>(reinterpret_cast<const unsigned long long *>(rowcnt.p), out.rp.p, nc + 1,
                                       nullptr, s);
    DBuf<unsigned long long> wsum;
    if (cols.size() == 1) {
        out.col = std::move(cols[0]);
        wsum = std::move(ws[0]);
    } else {
        out.col.alloc(U, s);
        wsum.alloc(U, s);
        int64_t at = 0;
        for (size_t r = 0; r < cols.size(); r++) {
            const int64_t u = (int64_t)cols[r].n;
            if (u) {
                CD_CUDA(cudaMemcpyAsync(out.col.p + at, cols[r].p, u * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                CD_CUDA(cudaMemcpyAsync(wsum.p + at, ws[r].p, u * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
            }
            cols[r].release();
            ws[r].release();
            at += u;
        }
    }
    if (big) {
        out.w64.alloc(U, s);
        if (U) CD_CUDA(cudaMemcpyAsync(out.w64.p, wsum.p, U * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        v.w = out.w64.p;
    } else {
        out.w32.alloc(U, s);
        if (U) { k_to_i32<<<grid_for(U, kBlock, 152 * 32), kBlock, 0, s>>>(wsum.p, U, out.w32.p); ::cd::note_launch(); }
        v.w = out.w32.p;
    }
    out.self.alloc(nc, s);
    if (nc) { k_finish_self<<<grid_for(nc, kBlock, 152 * 32), kBlock, 0, s>>>(intra2.p, nc, out.self.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    finish_graph(out, s);
}

}  // namespace cd
