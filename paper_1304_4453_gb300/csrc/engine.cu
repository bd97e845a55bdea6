// Host drivers: schedule construction, the move phase (Algorithm 2), PLP
// (Algorithm 1), the PLM / PLMR level loop (Algorithms 3, 4) and EPP
// (Algorithm 5).  Every step of the computation is a kernel; the host only
// sequences launches and reads back per-sweep counters.
#include <chrono>
#include <memory>

#include "engine.cuh"
#include "graph.cuh"
#include "move_dispatch.cuh"

namespace cd {

// Sweeps 0 .. RECHECK_FROM-1 of a move phase apply every wanted move of a
// class at once.  From sweep RECHECK_FROM on, a class's wanted moves are
// re-checked one by one in ascending vertex id against the volumes updated
// by the moves accepted before them (k_recheck), so every applied move raises
// modularity and the phase terminates.
constexpr int RECHECK_FROM = 4;

using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
}

// ---------------------------------------------------------------------------
// Schedule: vertices sorted by (colour, degree bin, id); degree-0 vertices
// form a trailing bucket that no kernel visits.
// ---------------------------------------------------------------------------
struct Schedule {
    int32_t ncol = 0;
    DBuf<int32_t> order;
    std::vector<int64_t> off;          // bucket k*NBINS+b -> [off[i], off[i+1])
    std::vector<int32_t> hub_start;    // per class, into the hub arrays
    std::vector<int32_t> nb1, nb2;     // per class H1 / H2 block totals
    DBuf<HubInfo> hubs;
    DBuf<int32_t> hb1, hb2;            // per hub, block prefix inside its class
    int64_t nhubs = 0, max_tab = 0, max_nb2 = 0;
    DBuf<int32_t> hub_keys;
    DBuf<unsigned long long> hub_vals, hub_wc;
    DBuf<unsigned int> done1, done2;
    DBuf<int64_t> part_g, part_g2, part_w;
    DBuf<int32_t> part_id;
    DBuf<uint32_t> part_tk;
    // class metadata on the device (persistent kernels)
    DBuf<int64_t> d_off;
    DBuf<int32_t> d_hub0, d_nb1, d_nb2;
};

__global__ void k_sched_keys(const int64_t *rp, int64_t n, const int32_t *color, int32_t ncol, uint32_t *key,
                             int32_t *val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        key[i] = d == 0 ? (uint32_t)ncol * NBINS : (uint32_t)color[i] * NBINS + degree_bin(d);
        val[i] = (int32_t)i;
    }
}

// off[b] = first position whose (sorted) key is >= b, for b in [0, nbk].
__global__ void k_bucket_bounds(const uint32_t *key, int64_t n, int64_t nbk, int64_t *off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = key[i];
        const int64_t kp = i == 0 ? -1 : (int64_t)key[i - 1];
        for (int64_t b = kp + 1; b <= k; b++) off[b] = i;
        if (i == n - 1)
            for (int64_t b = k + 1; b <= nbk; b++) off[b] = n;
    }
}

__global__ void k_degrees(const int64_t *rp, const int32_t *v, int64_t cnt, int64_t *deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        deg[i] = rp[v[i] + 1] - rp[v[i]];
}

static int bits_for(int64_t x) {
    int b = 1;
    while (((int64_t)1 << b) < x) b++;
    return b;
}

static void upload_class_meta(Schedule &S, cudaStream_t s) {
    S.d_off.alloc(S.off.size(), s);
    S.d_hub0.alloc(S.hub_start.size(), s);
    S.d_nb1.alloc(S.ncol + 1, s);
    S.d_nb2.alloc(S.ncol + 1, s);
    CD_CUDA(cudaMemcpyAsync(S.d_off.p, S.off.data(), S.off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CD_CUDA(cudaMemcpyAsync(S.d_hub0.p, S.hub_start.data(), S.hub_start.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
    if (S.ncol) {
        CD_CUDA(cudaMemcpyAsync(S.d_nb1.p, S.nb1.data(), S.ncol * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CD_CUDA(cudaMemcpyAsync(S.d_nb2.p, S.nb2.data(), S.ncol * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    CD_CUDA(cudaStreamSynchronize(s));   // the host vectors may change after return
}

static void build_schedule(const GraphView &g, uint64_t seed, Schedule &S, cudaStream_t s) {
    const int64_t n = g.n;
    DBuf<int32_t> color(n, s);
    S.ncol = color_graph(g, seed, color.p, s);
    const int64_t nbk = (int64_t)S.ncol * NBINS + 1;
    S.order.alloc(n, s);
    S.off.assign(nbk + 1, 0);
    if (n) {
        DBuf<uint32_t> key(n, s), key2(n, s);
        DBuf<int32_t> val2(n, s);
        { k_sched_keys<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(g.rp, n, color.p, S.ncol, key.p, S.order.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        std::vector<int> digits;
        for (int d = 0; d < bits_for(nbk + 1); d += 8) digits.push_back(d);
        radix_sort_pairs<uint32_t, int32_t>(key.p, S.order.p, key2.p, val2.p, n, digits, s);
        DBuf<int64_t> offd(nbk + 1, s);
        { k_bucket_bounds<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(key.p, n, nbk, offd.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        CD_CUDA(cudaMemcpyAsync(S.off.data(), offd.p, (nbk + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
    }
    // hubs, class by class
    S.hub_start.assign(S.ncol + 1, 0);
    S.nb1.assign(S.ncol, 0);
    S.nb2.assign(S.ncol, 0);
    int64_t H = 0;
    for (int32_t k = 0; k < S.ncol; k++) {
        S.hub_start[k] = (int32_t)H;
        H += S.off[(int64_t)k * NBINS + 5] - S.off[(int64_t)k * NBINS + 4];
    }
    S.hub_start[S.ncol] = (int32_t)H;
    S.nhubs = H;
    S.max_tab = S.max_nb2 = 0;
    if (H == 0) {
        upload_class_meta(S, s);
        return;
    }
    std::vector<int32_t> hv(H);
    std::vector<int64_t> hd(H);
    {
        Pinned pv(H * sizeof(int32_t)), pd(H * sizeof(int64_t));
        for (int32_t k = 0; k < S.ncol; k++) {
            const int64_t a = S.off[(int64_t)k * NBINS + 4], e = S.off[(int64_t)k * NBINS + 5];
            if (e > a)
                CD_CUDA(cudaMemcpyAsync(pv.as<int32_t>() + S.hub_start[k], S.order.p + a, (e - a) * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
        }
        CD_CUDA(cudaStreamSynchronize(s));
        DBuf<int32_t> dv(H, s);
        DBuf<int64_t> dd(H, s);
        CD_CUDA(cudaMemcpyAsync(dv.p, pv.p, H * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        { k_degrees<<<grid_for(H, kBlock), kBlock, 0, s>>>(g.rp, dv.p, H, dd.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        CD_CUDA(cudaMemcpyAsync(pd.p, dd.p, H * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < H; i++) { hv[i] = pv.as<int32_t>()[i]; hd[i] = pd.as<int64_t>()[i]; }
    }
    std::vector<HubInfo> info(H);
    std::vector<int32_t> b1(H), b2(H);
    for (int32_t k = 0; k < S.ncol; k++) {
        int64_t tab = 0;
        int32_t c1 = 0, c2 = 0;
        for (int32_t h = S.hub_start[k]; h < S.hub_start[k + 1]; h++) {
            int64_t slots = BLK_SLOTS;
            while (slots < 2 * hd[h]) slots <<= 1;
            HubInfo &x = info[h];
            x.v = hv[h];
            x.nb1 = (int32_t)((hd[h] + HUB_CHUNK - 1) / HUB_CHUNK);
            x.nb2 = (int32_t)((slots + HUB_SCAN - 1) / HUB_SCAN);
            x.pad = 0;
            x.tab = tab;
            x.slots = slots;
            b1[h] = c1;
            b2[h] = c2;
            c1 += x.nb1;
            c2 += x.nb2;
            tab += slots;
        }
        S.nb1[k] = c1;
        S.nb2[k] = c2;
        S.max_tab = std::max(S.max_tab, tab);
        S.max_nb2 = std::max<int64_t>(S.max_nb2, c2);
    }
    S.hubs.alloc(H, s);
    S.hb1.alloc(H, s);
    S.hb2.alloc(H, s);
    CD_CUDA(cudaMemcpyAsync(S.hubs.p, info.data(), H * sizeof(HubInfo), cudaMemcpyHostToDevice, s));
    CD_CUDA(cudaMemcpyAsync(S.hb1.p, b1.data(), H * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CD_CUDA(cudaMemcpyAsync(S.hb2.p, b2.data(), H * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    S.hub_keys.alloc(S.max_tab, s);
    CD_CUDA(cudaMemsetAsync(S.hub_keys.p, 0xff, S.max_tab * sizeof(int32_t), s));
    S.hub_vals.alloc(S.max_tab, s);
    S.hub_vals.zero();
    S.hub_wc.alloc(H, s);
    S.done1.alloc(H, s);
    S.done1.zero();
    S.done2.alloc(H, s);
    S.done2.zero();
    S.part_g.alloc(S.max_nb2, s);
    S.part_g2.alloc(S.max_nb2, s);
    S.part_w.alloc(S.max_nb2, s);
    S.part_id.alloc(S.max_nb2, s);
    S.part_tk.alloc(S.max_nb2, s);
    upload_class_meta(S, s);
    CD_CUDA(cudaStreamSynchronize(s));   // host vectors above go out of scope
}

static int wbytes(int wk) { return wk == W_UNIT ? 0 : wk == W_I32 ? 4 : 8; }

// ---------------------------------------------------------------------------
// Move phase (Algorithm 2) under the colour-class schedule.
// ---------------------------------------------------------------------------
// Arguments shared by the persistent kernels: graph, schedule, hub tables.
static PhaseArgs phase_args(const GraphView &g, const Schedule &S, int32_t *zeta) {
    PhaseArgs a{};
    a.g = g;
    a.zeta = zeta;
    a.order = S.order.p;
    a.ncol = S.ncol;
    a.class_off = S.d_off.p;
    a.class_hub0 = S.d_hub0.p;
    a.class_nb1 = S.d_nb1.p;
    a.class_nb2 = S.d_nb2.p;
    a.hubs = S.hubs.p;
    a.hb1 = S.hb1.p;
    a.hb2 = S.hb2.p;
    a.hub_keys = S.hub_keys.p;
    a.hub_vals = S.hub_vals.p;
    a.hub_wc = S.hub_wc.p;
    a.done1 = S.done1.p;
    a.done2 = S.done2.p;
    a.part_g = S.part_g.p;
    a.part_g2 = S.part_g2.p;
    a.part_w = S.part_w.p;
    a.part_id = S.part_id.p;
    a.part_tk = S.part_tk.p;
    return a;
}

// Reads a persistent run's result words and per-sweep counters.
static int32_t finish_phase(const DBuf<int32_t> &result, const DBuf<Counters> &cnt, const DBuf<GridBarrier> &bar,
                            int32_t *conv, std::vector<Counters> &per, cudaStream_t s) {
    Pinned hr(4 * sizeof(int32_t) + sizeof(GridBarrier));
    CD_CUDA(cudaMemcpyAsync(hr.p, result.p, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(hr.as<char>() + 4 * sizeof(int32_t), bar.p, sizeof(GridBarrier), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const GridBarrier *hb = reinterpret_cast<const GridBarrier *>(hr.as<char>() + 4 * sizeof(int32_t));
    if (hb->err) raise(CD_ETIMEOUT, "a grid barrier of the persistent kernel timed out");
    const int32_t runs = hr.as<int32_t>()[0];
    *conv = hr.as<int32_t>()[1];
    per.resize(runs);
    if (runs) CD_CUDA(cudaMemcpyAsync(per.data(), cnt.p, runs * sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    for (const Counters &c : per)
        if (c.overflow) raise(CD_ECUDA, "internal hash table overflow (%llu failed inserts)", c.overflow);
    return runs;
}

// ---------------------------------------------------------------------------
// Move phase (Algorithm 2) under the colour-class schedule: one persistent
// launch.  volc holds the community volumes of zeta on entry.
// ---------------------------------------------------------------------------
static int64_t move_phase(const GraphView &g, const Schedule &S, int32_t *zeta, int64_t *volc, const RunOpts &o,
                          RunStats &st, LaunchTimer &timer, cudaStream_t s) {
    const bool big = needs_big(g.W);
    const int64_t ncol = S.ncol;
    DBuf<int32_t> mv_u(g.n, s), mv_c(g.n, s), cd_(g.n, s);
    DBuf<int64_t> cwd(g.n, s), cwc(g.n, s), volb(g.n, s);
    DBuf<uint64_t> tmp_a(g.n, s), tmp_b(g.n, s);
    DBuf<unsigned long long> nmv(2 * ncol + 1, s), ncand(ncol + 1, s);
    DBuf<Counters> cnt(o.max_sweeps, s);
    DBuf<GridBarrier> bar(1, s);
    DBuf<int32_t> result(4, s);
    cnt.zero();
    bar.zero();
    result.zero();
    nmv.zero();
    if (g.n) CD_CUDA(cudaMemcpyAsync(volb.p, volc, g.n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    PhaseArgs a = phase_args(g, S, zeta);
    a.cnt = cnt.p;
    a.bar = bar.p;
    a.result = result.p;
    a.vol_a = volc;
    a.vol_b = volb.p;
    a.mv_u = mv_u.p;
    a.mv_c = mv_c.p;
    a.cd = cd_.p;
    a.cwd = cwd.p;
    a.cwc = cwc.p;
    a.nmv = nmv.p;
    a.ncand = ncand.p;
    a.tmp_a = tmp_a.p;
    a.tmp_b = tmp_b.p;
    int ubits = 1;
    while (((int64_t)1 << ubits) < g.n) ubits++;
    a.ubits = ubits;
    a.max_sweeps = o.max_sweeps;
    a.recheck_from = RECHECK_FROM;
    DBuf<unsigned long long> stage(3, s);
    stage.zero();
    if (timer.on) a.stage_ns = stage.p;
    timer.before(s);
    launch_move_phase(g.wk, big, a, s);
    timer.after(s);
    int32_t conv = 0;
    std::vector<Counters> per;
    const int32_t sweeps = finish_phase(result, cnt, bar, &conv, per, s);
    int64_t total = 0;
    for (const Counters &h : per) {
        st.sweeps++;
        st.moves += h.moved;
        st.entries += h.entries;
        st.candidates += h.candidates;
        st.decisions += h.decisions;
        total += h.moved;
        if (timer.on)
            st.k_bytes += 40.0 * h.decisions + (8.0 + wbytes(g.wk)) * h.entries + 8.0 * h.candidates + 12.0 * h.moved;
    }
    if (timer.on) {
        st.k_ms += timer.collect_ms();
        unsigned long long ns[3];
        CD_CUDA(cudaMemcpy(ns, stage.p, sizeof(ns), cudaMemcpyDeviceToHost));
        for (int i = 0; i < 3; i++) st.stage_ms[i] += ns[i] * 1e-6;
    }
    if (!conv) st.converged = 0;
    (void)sweeps;
    return total;
}

__global__ void k_prolong(int32_t *zeta, const int64_t *rank, const int32_t *up, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        zeta[i] = up[rank[zeta[i]]];
}

__global__ void k_comm_volumes(const int32_t *zeta, const int64_t *vol, int64_t n, int64_t *volc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(volc + zeta[i]), (unsigned long long)vol[i]);
}

struct Level {
    OwnedGraph own;
    GraphView g;
    Schedule S;
    DBuf<int32_t> zeta;
    DBuf<int64_t> rank;
};

void run_plm(const GraphView &g0, bool refine, const RunOpts &o, int32_t *labels, RunStats &st, cudaStream_t s) {
    const auto t_all = Clock::now();
    LaunchTimer timer;
    timer.on = o.profile;
    std::vector<std::unique_ptr<Level>> L;
    L.push_back(std::make_unique<Level>());
    L[0]->g = g0;
    for (int depth = 0;; depth++) {
        Level &lv = *L.back();
        const int64_t n = lv.g.n;
        auto t = Clock::now();
        build_schedule(lv.g, o.seed, lv.S, s);
        st.ms_color += ms_since(t);
        if (depth == 0 && st.colors0 < 0) st.colors0 = lv.S.ncol;
        lv.zeta.alloc(n, s);
        iota32(lv.zeta.p, n, s);
        DBuf<int64_t> volc(n, s);
        if (n) CD_CUDA(cudaMemcpyAsync(volc.p, lv.g.vol, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        t = Clock::now();
        const int64_t moved = move_phase(lv.g, lv.S, lv.zeta.p, volc.p, o, st, timer, s);
        st.ms_move += ms_since(t);
        if (moved == 0 || depth + 1 >= o.max_levels) break;
        t = Clock::now();
        lv.rank.alloc(n, s);
        auto nx = std::make_unique<Level>();
        coarsen_graph(lv.g, lv.zeta.p, lv.rank.p, nx->own, s);
        nx->g = nx->own.view;
        L.push_back(std::move(nx));
        st.ms_coarsen += ms_since(t);
    }
    st.levels += (int32_t)L.size();
    int64_t k = compact_labels(L.back()->zeta.p, L.back()->g.n, s);
    for (int d = (int)L.size() - 2; d >= 0; d--) {
        Level &lv = *L[d];
        const int64_t n = lv.g.n;
        if (n)
            { k_prolong<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(lv.zeta.p, lv.rank.p, L[d + 1]->zeta.p, n); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        if (refine) {
            DBuf<int64_t> volc(n, s);
            volc.zero();
            if (n) { k_comm_volumes<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(lv.zeta.p, lv.g.vol, n, volc.p); ::cd::note_launch(); }
            CD_LAUNCH_CHECK();
            auto t = Clock::now();
            move_phase(lv.g, lv.S, lv.zeta.p, volc.p, o, st, timer, s);
            st.ms_move += ms_since(t);
            k = compact_labels(lv.zeta.p, n, s);
        }
        L.pop_back();
    }
    if (g0.n)
        CD_CUDA(cudaMemcpyAsync(labels, L[0]->zeta.p, g0.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    CD_CUDA(cudaStreamSynchronize(s));
    st.k_launches += timer.launches;
    st.ncomm = (int32_t)k;
    st.ms_total += ms_since(t_all);
}

// ---------------------------------------------------------------------------
// PLP (Algorithm 1)
// ---------------------------------------------------------------------------
static void plp_iterate(const GraphView &g, const Schedule &S, const RunOpts &o, double theta, int32_t *zeta,
                        RunStats &st, LaunchTimer &timer, cudaStream_t s) {
    const bool big = needs_big(g.W);
    DBuf<uint8_t> active(g.n, s);
    if (g.n) CD_CUDA(cudaMemsetAsync(active.p, 1, g.n, s));
    iota32(zeta, g.n, s);
    DBuf<Counters> cnt(o.max_iters + 1, s);
    DBuf<GridBarrier> bar(1, s);
    DBuf<int32_t> result(4, s);
    cnt.zero();
    bar.zero();
    result.zero();
    PhaseArgs a = phase_args(g, S, zeta);
    a.cnt = cnt.p;
    a.bar = bar.p;
    a.result = result.p;
    a.active = active.p;
    a.seed = o.seed;
    a.theta = theta;
    a.max_iters = o.max_iters;
    timer.before(s);
    launch_plp_run(g.wk, big, a, s);
    timer.after(s);
    int32_t conv = 0;
    std::vector<Counters> per;
    const int32_t iters = finish_phase(result, cnt, bar, &conv, per, s);
    const int64_t listed = S.off[(int64_t)S.ncol * NBINS];
    for (const Counters &h : per) {
        st.moves += h.moved;
        st.entries += h.entries;
        st.candidates += h.candidates;
        st.decisions += h.decisions;
        if (timer.on)
            st.k_bytes += 5.0 * listed + 20.0 * h.decisions + (8.0 + wbytes(g.wk)) * h.entries + 4.0 * h.moved;
    }
    if (timer.on) st.k_ms += timer.collect_ms();
    st.iters += iters;
    if (!conv) st.converged = 0;
}

void run_plp(const GraphView &g, const RunOpts &o, double theta, int32_t *labels, RunStats &st, cudaStream_t s) {
    const auto t_all = Clock::now();
    LaunchTimer timer;
    timer.on = o.profile;
    Schedule S;
    auto t = Clock::now();
    build_schedule(g, o.seed, S, s);
    st.ms_color += ms_since(t);
    if (st.colors0 < 0) st.colors0 = S.ncol;
    t = Clock::now();
    plp_iterate(g, S, o, theta, labels, st, timer, s);
    st.ms_move += ms_since(t);
    st.ncomm = (int32_t)compact_labels(labels, g.n, s);
    st.levels = 1;
    st.k_launches += timer.launches;
    st.ms_total += ms_since(t_all);
}

// ---------------------------------------------------------------------------
// EPP (Algorithm 5) with the exact core communities of Eq. (2).
// ---------------------------------------------------------------------------
__global__ void k_pair_keys(const int32_t *core, const int32_t *z, int64_t n, uint64_t *key, int32_t *val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ((uint64_t)(uint32_t)core[i] << 32) | (uint32_t)z[i];
        val[i] = (int32_t)i;
    }
}

__global__ void k_scatter_rank(const int32_t *val, const int32_t *head, const int64_t *uidx, int64_t n,
                               int32_t *core) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        core[val[i]] = (int32_t)(uidx[i] + head[i] - 1);
}

__global__ void k_heads64(const uint64_t *keys, int64_t cnt, int32_t *head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_gather_core(const int32_t *zc, const int32_t *core, int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = zc[core[i]];
}

// core <- dense rank of (core, z) pairs in ascending order.
static void fold_core(int32_t *core, const int32_t *z, int64_t n, cudaStream_t s) {
    DBuf<uint64_t> key(n, s), key2(n, s);
    DBuf<int32_t> val(n, s), val2(n, s), head(n, s);
    DBuf<int64_t> uidx(n, s);
    const unsigned gb = grid_for(n, kBlock, 152 * 32);
    { k_pair_keys<<<gb, kBlock, 0, s>>>(core, z, n, key.p, val.p); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    std::vector<int> digits;
    const int b = bits_for(n);
    for (int d = 0; d < b; d += 8) digits.push_back(d);
    for (int d = 0; d < b; d += 8) digits.push_back(32 + d);
    radix_sort_pairs<uint64_t, int32_t>(key.p, val.p, key2.p, val2.p, n, digits, s);
    { k_heads64<<<gb, kBlock, 0, s>>>(key.p, n, head.p); ::cd::note_launch(); }
    exclusive_scan<int32_t>(head.p, uidx.p, n, nullptr, s);
    { k_scatter_rank<<<gb, kBlock, 0, s>>>(val.p, head.p, uidx.p, n, core); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
}

void run_epp(const GraphView &g, int b, bool final_refine, const RunOpts &o, double theta, int32_t *labels,
             RunStats &st, cudaStream_t s) {
    const auto t_all = Clock::now();
    const int64_t n = g.n;
    DBuf<int32_t> base((size_t)b * n, s), core(n, s);
    for (int i = 0; i < b; i++) {
        RunOpts oi = o;
        oi.seed = o.seed + (uint64_t)i;
        RunStats si;
        run_plp(g, oi, theta, base.p + (size_t)i * n, si, s);
        st.iters += si.iters;
        st.moves += si.moves;
        st.entries += si.entries;
        st.candidates += si.candidates;
        st.decisions += si.decisions;
        st.k_ms += si.k_ms;
        st.k_bytes += si.k_bytes;
        st.k_launches += si.k_launches;
        st.ms_color += si.ms_color;
        st.ms_move += si.ms_move;
        if (!si.converged) st.converged = 0;
        if (i == 0) st.colors0 = si.colors0;
    }
    if (n) {
        CD_CUDA(cudaMemcpyAsync(core.p, base.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        for (int i = 1; i < b; i++) fold_core(core.p, base.p + (size_t)i * n, n, s);
    }
    auto t = Clock::now();
    OwnedGraph cg;
    DBuf<int64_t> rank(n, s);
    coarsen_graph(g, core.p, rank.p, cg, s);
    st.ms_coarsen += ms_since(t);
    DBuf<int32_t> zc(cg.view.n, s);
    RunStats sf;
    run_plm(cg.view, final_refine, o, zc.p, sf, s);
    st.levels = sf.levels;
    st.sweeps += sf.sweeps;
    st.moves += sf.moves;
    st.entries += sf.entries;
    st.candidates += sf.candidates;
    st.decisions += sf.decisions;
    st.k_ms += sf.k_ms;
    st.k_bytes += sf.k_bytes;
    st.k_launches += sf.k_launches;
    for (int i = 0; i < 3; i++) st.stage_ms[i] += sf.stage_ms[i];
    st.ms_color += sf.ms_color;
    st.ms_move += sf.ms_move;
    st.ms_coarsen += sf.ms_coarsen;
    if (!sf.converged) st.converged = 0;
    if (n) { k_gather_core<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(zc.p, core.p, n, labels); ::cd::note_launch(); }
    CD_LAUNCH_CHECK();
    st.ncomm = (int32_t)compact_labels(labels, n, s);
    CD_CUDA(cudaStreamSynchronize(s));
    st.ms_total += ms_since(t_all);
}

}  // namespace cd
