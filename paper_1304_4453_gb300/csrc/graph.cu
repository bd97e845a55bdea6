// Graph construction: CSR validation, self-loop separation, vol(u) and
// omega(E) (Section III-B definitions), export back to input form.
#include "common.cuh"
#include "graph.cuh"

namespace cd {

enum {
    BAD_ROWPTR = 1, BAD_COL = 2, BAD_ORDER = 4, BAD_WEIGHT = 8, BAD_ASYM = 16, BAD_ASYMW = 32
};

// One warp per row: ranges, strict column order, positive weights, and the
// mirror entry (v, u) with the same weight for every (u, v), u != v.
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col, const int32_t *w,
                           int *err, int32_t *loops) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int64_t beg = rp[u], end = rp[u + 1];
        int bad = 0, nl = 0;
        if (beg < 0 || end > nnz || end < beg) {
            bad |= BAD_ROWPTR;
        } else {
            for (int64_t e = beg + lane; e < end; e += 32) {
                int32_t v = col[e];
                if (v < 0 || v >= n) { bad |= BAD_COL; continue; }
                if (e > beg && col[e - 1] >= v) bad |= BAD_ORDER;
                if (w && w[e] <= 0) bad |= BAD_WEIGHT;
                if (v == u) { nl++; continue; }
                int64_t lo = rp[v], hi = rp[v + 1];
                if (lo < 0 || hi > nnz || hi < lo) { bad |= BAD_ROWPTR; continue; }
                hi -= 1;
                int64_t pos = -1;
                while (lo <= hi) {
                    int64_t mid = lo + ((hi - lo) >> 1);
                    int32_t c = col[mid];
                    if (c == u) { pos = mid; break; }
                    if (c < u) lo = mid + 1; else hi = mid - 1;
                }
                if (pos < 0) bad |= BAD_ASYM;
                else if (w && w[pos] != w[e]) bad |= BAD_ASYMW;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
            nl += __shfl_xor_sync(0xffffffffu, nl, o);
        }
        if (lane == 0) {
            loops[u] = nl;
            if (bad) atomicOr(err, bad);
        }
    }
}

// Copies row u without its self-loop (at most one, rows being strictly sorted).
template <bool HASW>
__global__ void k_strip_loops(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                              const int64_t *loops_before, int64_t *nrp, int32_t *ncol, int32_t *nw, int64_t *self) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int64_t beg = rp[u], end = rp[u + 1];
        int64_t out = beg - loops_before[u];
        if (lane == 0) { nrp[u] = out; self[u] = 0; }
        if (u == n - 1 && lane == 0) nrp[n] = end - loops_before[n];
        // find the loop position (if any)
        int64_t lp = end;
        for (int64_t e = beg + lane; e < end; e += 32)
            if (col[e] == u) lp = e;
        for (int o = 16; o > 0; o >>= 1) lp = min(lp, __shfl_xor_sync(0xffffffffu, lp, o));
        for (int64_t e = beg + lane; e < end; e += 32) {
            if (e == lp) {
                self[u] = HASW ? (int64_t)w[e] : 1;
                continue;
            }
            int64_t o2 = out + (e - beg) - (e > lp ? 1 : 0);
            ncol[o2] = col[e];
            if (HASW) nw[o2] = w[e];
        }
    }
}

// vol(u) = sum of weights to other vertices + 2 * self-loop; block sums of vol
// (= 2 omega(E)) and of max degree.
__global__ void k_volumes(int64_t n, const int64_t *rp, const void *w, int wk, const int64_t *self,
                          int64_t *vol, unsigned long long *twoW, unsigned long long *maxdeg) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t acc = 0, md = 0;
    for (int64_t u = warp; u < n; u += nwarps) {
        int64_t beg = rp[u], end = rp[u + 1];
        int64_t s = 0;
        if (wk == W_UNIT) {
            s = end - beg;
        } else {
            for (int64_t e = beg + lane; e < end; e += 32) s += edge_weight_rt(w, wk, e);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        s += 2 * self[u];
        if (lane == 0) vol[u] = s;
        acc += s;
        md = max(md, end - beg);
    }
    if (lane == 0) {
        atomicAdd(twoW, (unsigned long long)acc);
        atomicMax(maxdeg, (unsigned long long)md);
    }
}

void finish_graph(OwnedGraph &g, cudaStream_t s, bool borrowed) {
    GraphView &v = g.view;
    if (!borrowed) {   // else rp and col already point at the caller's arrays
        v.rp = g.rp.p;
        v.col = g.col.p;
    }
    v.self = g.self.p;
    g.vol.alloc(v.n, s);
    v.vol = g.vol.p;
    v.W = 0;
    v.max_deg = 0;
    if (v.n == 0) return;
    DBuf<unsigned long long> red(2, s);
    red.zero();
    { k_volumes<<<grid_for(v.n * 32, kBlock, 152 * 64), kBlock, 0, s>>>(v.n, v.rp, v.w, v.wk, v.self, g.vol.p,
                                                                     red.p, red.p + 1); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    Pinned h(2 * sizeof(unsigned long long));
    CD_CUDA(cudaMemcpyAsync(h.p, red.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    v.W = (int64_t)(h.as<unsigned long long>()[0] / 2);
    v.max_deg = (int64_t)h.as<unsigned long long>()[1];
}

void build_graph(int64_t n, const int64_t *rp_in, const int32_t *col_in, const int32_t *w_in, int mem,
                 cudaStream_t s, OwnedGraph &out) {
    if (n < 0 || n >= ((int64_t)1 << 31)) raise(CD_EINVAL, "n = %lld out of range [0, 2^31)", (long long)n);
    if (!rp_in) raise(CD_EINVAL, "row_ptr is NULL");
    int64_t first = 0, nnz = 0;
    if (mem == CD_MEM_HOST) {
        first = rp_in[0];
        nnz = rp_in[n];
    } else if (mem == CD_MEM_DEVICE || mem == CD_BORROW) {
        CD_CUDA(cudaMemcpy(&first, rp_in, sizeof(int64_t), cudaMemcpyDeviceToHost));
        CD_CUDA(cudaMemcpy(&nnz, rp_in + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
        raise(CD_EINVAL, "unknown memory flag %d", mem);
    }
    if (first != 0 || nnz < 0) raise(CD_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
    if (nnz > 0 && !col_in) raise(CD_EINVAL, "col is NULL");
    const bool borrow = mem == CD_BORROW;
    cudaMemcpyKind kind = mem == CD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;

    // staging copies of the input (borrowed arrays are read in place)
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<int32_t> w;
    const int64_t *rp_d = rp_in;
    const int32_t *col_d = col_in, *w_d = w_in;
    if (!borrow) {
        rp.alloc(n + 1, s);
        col.alloc(nnz, s);
        CD_CUDA(cudaMemcpyAsync(rp.p, rp_in, (n + 1) * sizeof(int64_t), kind, s));
        if (nnz) CD_CUDA(cudaMemcpyAsync(col.p, col_in, nnz * sizeof(int32_t), kind, s));
        if (w_in) {
            w.alloc(nnz, s);
            if (nnz) CD_CUDA(cudaMemcpyAsync(w.p, w_in, nnz * sizeof(int32_t), kind, s));
        }
        rp_d = rp.p;
        col_d = col.p;
        w_d = w_in ? w.p : nullptr;
    }
    DBuf<int> err(1, s);
    err.zero();
    DBuf<int32_t> loops(n + 1, s);
    if (n) {
        { k_validate<<<grid_for(n * 32, kBlock, 152 * 64), kBlock, 0, s>>>(n, nnz, rp_d, col_d, w_d,
                                                                        err.p, loops.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
    }
    DBuf<int64_t> loops_before(n + 1, s);
    CD_CUDA(cudaMemsetAsync(loops.p + n, 0, sizeof(int32_t), s));
    exclusive_scan<int32_t>(loops.p, loops_before.p, n + 1, nullptr, s);
    Pinned h(2 * sizeof(int64_t));
    CD_CUDA(cudaMemcpyAsync(h.p, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(h.as<int64_t>() + 1, loops_before.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    int bad = *h.as<int>();
    if (bad) {
        const char *why = (bad & BAD_ROWPTR) ? "row_ptr not monotone or out of range"
                        : (bad & BAD_COL) ? "column index out of range"
                        : (bad & BAD_ORDER) ? "row not strictly ascending (unsorted or duplicate column)"
                        : (bad & BAD_WEIGHT) ? "non-positive weight"
                        : (bad & BAD_ASYM) ? "asymmetric entry (missing mirror (v,u))"
                        : "asymmetric weight";
        raise(CD_EINVAL, "invalid CSR: %s", why);
    }
    int64_t nloops = h.as<int64_t>()[1];
    int64_t m_nnz = nnz - nloops;

    GraphView &v = out.view;
    v = GraphView();
    v.n = n;
    v.nnz = m_nnz;
    v.wk = w_in ? W_I32 : W_UNIT;
    out.self.alloc(n, s);
    bool borrowed = false;
    if (nloops == 0 && borrow) {
        v.rp = rp_d;
        v.col = col_d;
        v.w = w_d;
        out.self.zero();
        borrowed = true;
    } else if (nloops == 0) {
        out.rp = std::move(rp);
        out.col = std::move(col);
        if (w_in) out.w32 = std::move(w);
        out.self.zero();
    } else {
        out.rp.alloc(n + 1, s);
        out.col.alloc(m_nnz, s);
        if (w_in) out.w32.alloc(m_nnz, s);
        unsigned gb = grid_for(n * 32, kBlock, 152 * 64);
        if (w_in)
            { k_strip_loops<true><<<gb, kBlock, 0, s>>>(n, rp_d, col_d, w_d, loops_before.p, out.rp.p, out.col.p,
                                                     out.w32.p, out.self.p); ::cd::note_launch(); }
        else
            { k_strip_loops<false><<<gb, kBlock, 0, s>>>(n, rp_d, col_d, nullptr, loops_before.p, out.rp.p, out.col.p,
                                                      nullptr, out.self.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
    }
    if (!borrowed) v.w = w_in ? (const void *)out.w32.p : nullptr;
    finish_graph(out, s, borrowed);
}

// ---------------------------------------------------------------------------
// Export in input form (self-loop once, in sorted position).
// ---------------------------------------------------------------------------
__global__ void k_loop_flags(int64_t n, const int64_t *self, int32_t *f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = self[i] > 0 ? 1 : 0;
}

__global__ void k_export(GraphView g, const int64_t *loops_before, int64_t *orp, int32_t *ocol, int64_t *ow) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < g.n; u += nwarps) {
        int64_t beg = g.rp[u], end = g.rp[u + 1];
        int64_t out = beg + loops_before[u];
        bool has = g.self[u] > 0;
        // number of neighbours below u decides the loop slot
        int64_t below = 0;
        for (int64_t e = beg + lane; e < end; e += 32) below += g.col[e] < u ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
        if (lane == 0) {
            if (orp) orp[u] = out;
            if (orp && u == g.n - 1) orp[g.n] = end + loops_before[u] + (has ? 1 : 0);
            if (has && ocol) { ocol[out + below] = (int32_t)u; ow[out + below] = g.self[u]; }
        }
        if (!ocol) continue;
        for (int64_t e = beg + lane; e < end; e += 32) {
            int64_t k = e - beg;
            int64_t o2 = out + k + ((has && k >= below) ? 1 : 0);
            ocol[o2] = g.col[e];
            ow[o2] = edge_weight_rt(g.w, g.wk, e);
        }
    }
}

int64_t export_graph(const GraphView &g, int64_t *rp, int32_t *col, int64_t *w, int mem, cudaStream_t s) {
    DBuf<int32_t> f(g.n + 1, s);
    DBuf<int64_t> lb(g.n + 1, s);
    CD_CUDA(cudaMemsetAsync(f.p, 0, (g.n + 1) * sizeof(int32_t), s));
    if (g.n) { k_loop_flags<<<grid_for(g.n, kBlock, 152 * 32), kBlock, 0, s>>>(g.n, g.self, f.p); ::cd::note_launch(); }
    exclusive_scan<int32_t>(f.p, lb.p, g.n + 1, nullptr, s);
    Pinned h(sizeof(int64_t));
    CD_CUDA(cudaMemcpyAsync(h.p, lb.p + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    int64_t nnz = g.nnz + *h.as<int64_t>();
    if (!rp && !col && !w) return nnz;
    bool dev = mem == CD_MEM_DEVICE;
    DBuf<int64_t> drp, dw;
    DBuf<int32_t> dcol;
    int64_t *orp = rp, *ow = w;
    int32_t *ocol = col;
    if (!dev) {
        if (rp) { drp.alloc(g.n + 1, s); orp = drp.p; }
        if (col) { dcol.alloc(nnz, s); ocol = dcol.p; dw.alloc(nnz, s); ow = dw.p; }
    }
    if (col && !w && dev) raise(CD_EINVAL, "export needs col and w together");
    if (g.n == 0) {
        if (orp) CD_CUDA(cudaMemsetAsync(orp, 0, sizeof(int64_t), s));
    } else {
        { k_export<<<grid_for(g.n * 32, kBlock, 152 * 64), kBlock, 0, s>>>(g, lb.p, orp, col ? ocol : nullptr,
                                                                        col ? ow : nullptr); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
    }
    if (!dev) {
        if (rp) CD_CUDA(cudaMemcpyAsync(rp, orp, (g.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (col) CD_CUDA(cudaMemcpyAsync(col, ocol, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (col && w) CD_CUDA(cudaMemcpyAsync(w, ow, nnz * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    CD_CUDA(cudaStreamSynchronize(s));
    return nnz;
}

}  // namespace cd
