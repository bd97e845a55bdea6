// Host engine: schedule construction, the move phase (Algorithm 2), PLP
// (Algorithm 1), the PLM / PLMR level loop (Algorithms 3, 4) and EPP
// (Algorithm 5) as jobs that advance on host worker threads and meet in
// batched persistent launches.  Every step of the computation is a kernel;
// the host only sequences launches and reads back per-sweep counters.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>

#include "engine.cuh"
#include "graph.cuh"
#include "move_dispatch.cuh"

namespace cd {

// Sweeps 0 .. RECHECK_FROM-1 of a move phase apply every wanted move of a
// class at once.  From sweep RECHECK_FROM on, a class's wanted moves are
// re-checked one by one in ascending vertex id against the volumes updated
// by the moves accepted before them (the re-check), so every applied move raises
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
    std::vector<int32_t> nrelax;       // per class, hubs with more than HUB_RELAX neighbours
    DBuf<HubInfo> hubs;
    DBuf<int32_t> hb1, hb2;            // per hub, block prefix inside its class
    DBuf<ChunkDesc> chunks;            // aggregation items, class by class
    DBuf<SliceDesc> slices;            // decide slices, class by class
    DBuf<ClassMeta> meta;              // per class
    DBuf<int32_t> hub_occ;             // occupied-slot lists (laid out like hub_keys)
    DBuf<unsigned int> hub_nocc;
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

__global__ void k_sched_keys(const int64_t *rp, int64_t n, const int32_t *color, int32_t ncol, BinLimits bins,
                             uint32_t *key, int32_t *val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        key[i] = d == 0 ? (uint32_t)ncol * NBINS : (uint32_t)color[i] * NBINS + degree_bin(d, bins);
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

__global__ void k_rows(const int64_t *rp, const int32_t *v, int64_t cnt, int64_t *beg, int64_t *deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        beg[i] = rp[v[i]];
        deg[i] = rp[v[i] + 1] - rp[v[i]];
    }
}

static int bits_for(int64_t x) {
    int b = 1;
    while (((int64_t)1 << b) < x) b++;
    return b;
}

static void upload_class_meta(Schedule &S, const std::vector<int32_t> &it0, const std::vector<int32_t> &sl0,
                              cudaStream_t s) {
    std::vector<ClassMeta> meta(S.ncol);
    for (int32_t k = 0; k < S.ncol; k++) {
        ClassMeta &m = meta[k];
        m = ClassMeta{};
        for (int b = 0; b <= NBINS; b++) m.off[b] = S.off[(int64_t)k * NBINS + b];
        m.h0 = S.hub_start[k];
        m.nhubs = S.hub_start[k + 1] - S.hub_start[k];
        m.nb1 = S.nb1[k];
        m.nb2 = S.nb2[k];
        m.it0 = it0[k];
        m.sl0 = sl0[k];
        m.nrelax = S.nrelax.empty() ? 0 : S.nrelax[k];
    }
    S.meta.alloc(S.ncol, s);
    if (S.ncol)
        CD_CUDA(cudaMemcpyAsync(S.meta.p, meta.data(), S.ncol * sizeof(ClassMeta), cudaMemcpyHostToDevice, s));
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

__global__ void k_hash_rounds(int64_t n, uint32_t salt, int32_t rounds, int32_t *color) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        color[i] = (int32_t)(fmix32((uint32_t)i ^ salt) % (uint32_t)rounds);
}

// racy > 0: no colouring; the vertices are split into `racy` rounds by a
// seeded hash, adjacent vertices may share a round (the paper's parallel
// loop on live data, Section III-B, with the loop cut into rounds so that a
// vertex sees the moves of earlier rounds).
static void build_schedule(const GraphView &g, uint64_t seed, const BinLimits &bins, Schedule &S, cudaStream_t s,
                           int32_t racy = 0) {
    const int64_t n = g.n;
    DBuf<int32_t> color(n, s);
    if (racy > 0) {
        if (n) { k_hash_rounds<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(n, fmix32(seed_word(seed) ^ 0x52414359u), racy, color.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        S.ncol = n ? racy : 0;
    } else {
        S.ncol = color_graph(g, seed, color.p, s);
    }
    const int64_t nbk = (int64_t)S.ncol * NBINS + 1;
    S.order.alloc(n, s);
    S.off.assign(nbk + 1, 0);
    if (n) {
        DBuf<uint32_t> key(n, s), key2(n, s);
        DBuf<int32_t> val2(n, s);
        { k_sched_keys<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(g.rp, n, color.p, S.ncol, bins, key.p, S.order.p); ::cd::note_launch(); }
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
    S.nrelax.assign(S.ncol, 0);
    int64_t H = 0;
    for (int32_t k = 0; k < S.ncol; k++) {
        S.hub_start[k] = (int32_t)H;
        H += S.off[(int64_t)k * NBINS + 6] - S.off[(int64_t)k * NBINS + 5];   // hub-path bucket
    }
    S.hub_start[S.ncol] = (int32_t)H;
    S.nhubs = H;
    S.max_tab = S.max_nb2 = 0;
    if (H == 0) {
        upload_class_meta(S, std::vector<int32_t>(S.ncol + 1, 0), std::vector<int32_t>(S.ncol + 1, 0), s);
        return;
    }
    std::vector<int32_t> hv(H);
    std::vector<int64_t> hd(H), hb(H);
    {
        Pinned pv(H * sizeof(int32_t)), pd(2 * H * sizeof(int64_t));
        for (int32_t k = 0; k < S.ncol; k++) {
            const int64_t a = S.off[(int64_t)k * NBINS + 5], e = S.off[(int64_t)k * NBINS + 6];
            if (e > a)
                CD_CUDA(cudaMemcpyAsync(pv.as<int32_t>() + S.hub_start[k], S.order.p + a, (e - a) * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
        }
        CD_CUDA(cudaStreamSynchronize(s));
        DBuf<int32_t> dv(H, s);
        DBuf<int64_t> dd(2 * H, s);
        CD_CUDA(cudaMemcpyAsync(dv.p, pv.p, H * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        { k_rows<<<grid_for(H, kBlock), kBlock, 0, s>>>(g.rp, dv.p, H, dd.p, dd.p + H); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        CD_CUDA(cudaMemcpyAsync(pd.p, dd.p, 2 * H * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CD_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < H; i++) {
            hv[i] = pv.as<int32_t>()[i];
            hb[i] = pd.as<int64_t>()[i];
            hd[i] = pd.as<int64_t>()[H + i];
        }
    }
    std::vector<HubInfo> info(H);
    std::vector<int32_t> b1(H), b2(H);
    std::vector<int32_t> it0(S.ncol + 1, 0), sl0(S.ncol + 1, 0);
    std::vector<ChunkDesc> chunks;
    std::vector<SliceDesc> slices;
    for (int32_t k = 0; k < S.ncol; k++) {
        int64_t tab = 0;
        int32_t c1 = 0, c2 = 0;
        it0[k] = (int32_t)chunks.size();
        sl0[k] = (int32_t)slices.size();
        for (int32_t h = S.hub_start[k]; h < S.hub_start[k + 1]; h++) {
            int64_t slots = BLK_SLOTS;
            while (slots < 2 * hd[h]) slots <<= 1;
            HubInfo &x = info[h];
            x.v = hv[h];
            x.nb1 = (int32_t)((hd[h] + HUB_CHUNK - 1) / HUB_CHUNK);
            // hubs up to HUB_LAST are decided by their last aggregation item
            // (the occupied list of a hub holds at most deg entries)
            x.nb2 = hd[h] <= HUB_LAST ? 0 : (int32_t)((hd[h] + HUB_SCAN - 1) / HUB_SCAN);
            x.pad = 0;
            x.tab = tab;
            x.slots = slots;
            const int32_t hr = h - S.hub_start[k];
            for (int32_t j = 0; j < x.nb1; j++) {
                ChunkDesc d{};
                d.beg = hb[h] + (int64_t)j * HUB_CHUNK;
                d.end = std::min(hb[h] + hd[h], d.beg + HUB_CHUNK);
                d.tab = tab;
                d.slots = slots;
                d.u = hv[h];
                d.h = hr;
                d.nb1 = x.nb1;
                d.nb2 = x.nb2;
                d.relax = hd[h] > HUB_RELAX;
                chunks.push_back(d);
            }
            for (int32_t j = 0; j < x.nb2; j++) {
                SliceDesc d{};
                d.tab = tab;
                d.s0 = (int64_t)j * HUB_SCAN;
                d.s1 = d.s0 + HUB_SCAN;
                d.u = hv[h];
                d.h = hr;
                d.nb1 = x.nb1;
                d.nb2 = x.nb2;
                d.p0 = c2;
                d.relax = hd[h] > HUB_RELAX;
                slices.push_back(d);
            }
            if (hd[h] > HUB_RELAX) S.nrelax[k]++;
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
    it0[S.ncol] = (int32_t)chunks.size();
    sl0[S.ncol] = (int32_t)slices.size();
    S.chunks.alloc(chunks.size(), s);
    S.slices.alloc(slices.size(), s);
    if (!chunks.empty())
        CD_CUDA(cudaMemcpyAsync(S.chunks.p, chunks.data(), chunks.size() * sizeof(ChunkDesc), cudaMemcpyHostToDevice, s));
    if (!slices.empty())
        CD_CUDA(cudaMemcpyAsync(S.slices.p, slices.data(), slices.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice,
                                s));
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
    S.hub_wc.zero();   // omega(u, C) slots: written by a decide slice, reset by the last one
    S.hub_occ.alloc(S.max_tab, s);
    S.hub_nocc.alloc(H, s);
    S.hub_nocc.zero();
    S.done1.alloc(H, s);
    S.done1.zero();
    S.done2.alloc(H, s);
    S.done2.zero();
    S.part_g.alloc(S.max_nb2, s);
    S.part_g2.alloc(S.max_nb2, s);
    S.part_w.alloc(S.max_nb2, s);
    S.part_id.alloc(S.max_nb2, s);
    S.part_tk.alloc(S.max_nb2, s);
    upload_class_meta(S, it0, sl0, s);
    CD_CUDA(cudaStreamSynchronize(s));   // host vectors above go out of scope
}

static int wbytes(int wk) { return wk == W_UNIT ? 0 : wk == W_I32 ? 4 : 8; }

// ---------------------------------------------------------------------------
// Persistent phases.  A PhaseRun owns the buffers and arguments of one PLM
// move phase (Algorithm 2) or one PLP run (Algorithm 1) of one graph.
// ---------------------------------------------------------------------------
struct PhaseRun {
    bool plp = false;
    int wk = W_UNIT;
    bool big = false;
    bool profile = false;
    int64_t work = 0;             // adjacency entries + vertices (team sizing)
    int64_t quantum = 1;          // launch shape (RunOpts::team_quantum, team_min)
    int32_t team_min = 1;
    int64_t listed = 0;           // vertices the schedule visits
    int32_t cap = 0;              // counter slots
    PhaseArgs a{};
    DBuf<Counters> cnt;           // cap counters, then one slot holding the result words
    DBuf<unsigned long long> stage;
    DBuf<int32_t> mv_u, mv_c, cd_;
    DBuf<int64_t> vol_a, vol_b, cwd, cwc;
    DBuf<uint64_t> tmp_a, tmp_b;
    DBuf<int32_t> rc_u;               // re-check records in id order
    DBuf<uint64_t> rc_cd, rc_vu;
    DBuf<int64_t> rc_dw;
    DBuf<unsigned long long> nmv, ncand;
    DBuf<uint8_t> active;
    DBuf<unsigned long long> sched;   // decide-slice and class-finish counters
    DBuf<int32_t> dz_u, dz_l;         // deferred hub labels
    DBuf<int32_t> cstamp;             // re-check community stamps
    DBuf<unsigned int> dz_n;
    // class trace (RunOpts::trace): timestamps and the per-class sizes
    DBuf<unsigned long long> cls_ns, cls_stage;
    std::vector<int64_t> cls_info;    // per class: vertices, entries, hub chunks, hub slices, relaxed hubs
    // set by the engine after the launch
    double launch_ms = 0, wall_ms = 0;
    cd_status fail = CD_OK;
    std::string fail_msg;
};

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
    a.chunks = S.chunks.p;
    a.slices = S.slices.p;
    a.meta = S.meta.p;
    a.hub_occ = S.hub_occ.p;
    a.hub_nocc = S.hub_nocc.p;
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

static void alloc_counters(PhaseRun &r, int32_t cap, int64_t nhubs, int64_t n, cudaStream_t s) {
    r.sched.alloc(2, s);
    r.sched.zero();
    r.a.sched = r.sched.p;
    r.dz_u.alloc(nhubs + 1, s);
    r.dz_l.alloc(nhubs + 1, s);
    r.cstamp.alloc(n, s);
    r.cstamp.zero();
    r.dz_n.alloc(1, s);
    r.dz_n.zero();
    r.a.dz_u = r.dz_u.p;
    r.a.dz_l = r.dz_l.p;
    r.a.dz_n = r.dz_n.p;
    r.a.cstamp = r.cstamp.p;
    r.cap = cap;
    r.cnt.alloc((size_t)cap + 1, s);
    r.cnt.zero();
    r.a.cnt = r.cnt.p;
    r.a.result = reinterpret_cast<int32_t *>(r.cnt.p + cap);
    if (r.profile) {
        r.stage.alloc(3, s);
        r.stage.zero();
        r.a.stage_ns = r.stage.p;
    }
}

// Reads a finished run's result words and per-sweep counters.
static int32_t read_counters(PhaseRun &r, int32_t *conv, std::vector<Counters> &per, RunStats &st, cudaStream_t s) {
    if (r.fail != CD_OK) raise(r.fail, "%s", r.fail_msg.c_str());
    per.resize((size_t)r.cap + 1);
    CD_CUDA(cudaMemcpyAsync(per.data(), r.cnt.p, per.size() * sizeof(Counters), cudaMemcpyDeviceToHost, s));
    unsigned long long ns[3] = {0, 0, 0};
    if (r.profile) CD_CUDA(cudaMemcpyAsync(ns, r.stage.p, sizeof(ns), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const int32_t *res = reinterpret_cast<const int32_t *>(&per[r.cap]);
    const int32_t runs = res[0];
    *conv = res[1];
    if (runs < 0 || runs > r.cap) raise(CD_ECUDA, "persistent phase reported %d sweeps (cap %d)", runs, r.cap);
    per.resize(runs);
    for (const Counters &c : per)
        if (c.overflow) raise(CD_ECUDA, "internal hash table overflow (%llu failed inserts)", c.overflow);
    for (int i = 0; i < 3; i++) st.stage_ms[i] += ns[i] * 1e-6;
    st.ms_move += r.wall_ms;
    if (r.profile) {
        st.k_ms += r.launch_ms;
        st.k_launches += 1;
    }
    return runs;
}

// ---------------------------------------------------------------------------
// Class trace (profile level 2): per class step of a move phase, its wall time
// on block 0 from the previous class's barrier to its own, beside the class's
// size.  Diagnostic only; host copies of the schedule are made here.
// ---------------------------------------------------------------------------
static std::mutex g_trace_mu;
static std::vector<int64_t> g_trace;
static int64_t g_trace_phase = 0;

static void prepare_trace(PhaseRun &r, const GraphView &g, const Schedule &S, cudaStream_t s) {
    const int64_t ncol = S.ncol;
    r.cls_ns.alloc((size_t)r.cap * ncol + 1, s);
    r.cls_ns.zero();
    r.a.class_ns = r.cls_ns.p;
    r.cls_stage.alloc((size_t)r.cap * ncol * STAGE_SLOTS + 1, s);
    r.cls_stage.zero();
    r.a.stage_max = r.cls_stage.p;
    const int64_t listed = S.off[(size_t)ncol * NBINS];
    std::vector<int32_t> order((size_t)listed);
    std::vector<int64_t> rp((size_t)g.n + 1);
    if (listed) CD_CUDA(cudaMemcpyAsync(order.data(), S.order.p, listed * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(rp.data(), g.rp, ((size_t)g.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    r.cls_info.assign((size_t)ncol * 5, 0);
    for (int64_t k = 0; k < ncol; k++) {
        const int64_t a = S.off[(size_t)k * NBINS], b = S.off[(size_t)(k + 1) * NBINS];
        int64_t e = 0;
        for (int64_t i = a; i < b; i++) e += rp[order[i] + 1] - rp[order[i]];
        int64_t *ci = &r.cls_info[(size_t)k * 5];
        ci[0] = b - a;
        ci[1] = e;
        ci[2] = S.nb1[k];
        ci[3] = S.nb2[k];
        ci[4] = S.nrelax[k];
    }
}

static void record_trace(PhaseRun &r, int32_t runs, cudaStream_t s) {
    const int64_t ncol = r.a.ncol;
    std::vector<unsigned long long> t((size_t)runs * ncol + 1), sm((size_t)runs * ncol * STAGE_SLOTS + 1);
    CD_CUDA(cudaMemcpyAsync(t.data(), r.cls_ns.p, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaMemcpyAsync(sm.data(), r.cls_stage.p, sm.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            s));
    CD_CUDA(cudaStreamSynchronize(s));
    std::lock_guard<std::mutex> lk(g_trace_mu);
    const int64_t ph = g_trace_phase++;
    unsigned long long prev = t[0];
    for (int64_t sw = 0; sw < runs; sw++)
        for (int64_t k = 0; k < ncol; k++) {
            const unsigned long long x = t[1 + sw * ncol + k];
            if (x == 0) continue;
            const int64_t *ci = &r.cls_info[(size_t)k * 5];
            const unsigned long long *q = &sm[(size_t)(sw * ncol + k) * STAGE_SLOTS];
            // stage ends relative to the class start (0: the stage did not run)
            auto rel = [&](unsigned long long y) { return y > prev ? (int64_t)(y - prev) : (int64_t)0; };
            const int64_t row[TRACE_FIELDS] = {ph, sw, k, ci[0], ci[1], ci[2], ci[3], ci[4], (int64_t)(x - prev),
                                               rel(q[ST_ITEMS_END]), rel(q[ST_DECIDE_END]), rel(q[ST_FINISH_END]),
                                               rel(q[ST_FIRST_ITEM]), (int64_t)q[ST_GROUP], (int64_t)q[ST_BLOCK],
                                               (int64_t)q[ST_CHUNK], (int64_t)q[ST_SLICE_WAIT], (int64_t)q[ST_SLICE],
                                               (int64_t)q[ST_MOVES]};
            g_trace.insert(g_trace.end(), row, row + TRACE_FIELDS);
            prev = x;
        }
}

std::vector<int64_t> take_class_trace() {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    std::vector<int64_t> out;
    out.swap(g_trace);
    g_trace_phase = 0;
    return out;
}

__global__ void k_comm_volumes(const int32_t *zeta, const int64_t *vol, int64_t n, int64_t *volc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(volc + zeta[i]), (unsigned long long)vol[i]);
}

// Move phase of zeta on g.  init_vol: community volumes of zeta (the vertex
// volumes when zeta is the singleton partition); nullptr computes them.
static std::unique_ptr<PhaseRun> prepare_move(const GraphView &g, const Schedule &S, int32_t *zeta,
                                              const int64_t *init_vol, const RunOpts &o, cudaStream_t s) {
    auto r = std::make_unique<PhaseRun>();
    const int64_t n = g.n, ncol = S.ncol;
    r->plp = false;
    r->wk = g.wk;
    if (!gain_fits_128(g.W, o.res_p, o.res_q))
        raise(CD_EINVAL, "resolution %lld / %lld: max(p, q) (2W)^2 reaches 2^126 for 2W = %lld",
              (long long)o.res_p, (long long)o.res_q, (long long)(2 * g.W));
    r->big = o.int_path == 128 || gain_needs_big(g.W, o.res_p, o.res_q);
    if (o.int_path == 64 && r->big)
        raise(CD_EINVAL, "int_path 64: the gains of this graph and resolution need 128 bits");
    r->profile = o.profile;
    r->work = g.nnz + n;
    r->quantum = o.team_quantum;
    r->team_min = o.team_min;
    r->a = phase_args(g, S, zeta);
    r->mv_u.alloc(n, s);
    r->mv_c.alloc(n, s);
    r->cd_.alloc(n, s);
    r->cwd.alloc(n, s);
    r->cwc.alloc(n, s);
    r->vol_a.alloc(n, s);
    r->vol_b.alloc(n, s);
    r->tmp_a.alloc(n, s);
    r->tmp_b.alloc(n, s);
    r->rc_u.alloc(n, s);
    r->rc_cd.alloc(n, s);
    r->rc_vu.alloc(n, s);
    r->rc_dw.alloc(n, s);
    r->nmv.alloc(2 * ncol + 1, s);
    r->nmv.zero();
    r->ncand.alloc(ncol + 1, s);
    if (init_vol) {
        if (n) CD_CUDA(cudaMemcpyAsync(r->vol_a.p, init_vol, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    } else {
        r->vol_a.zero();
        if (n) { k_comm_volumes<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(zeta, g.vol, n, r->vol_a.p); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
    }
    if (n) CD_CUDA(cudaMemcpyAsync(r->vol_b.p, r->vol_a.p, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    alloc_counters(*r, o.max_sweeps, S.nhubs, n, s);
    PhaseArgs &a = r->a;
    a.vol_a = r->vol_a.p;
    a.vol_b = r->vol_b.p;
    a.mv_u = r->mv_u.p;
    a.mv_c = r->mv_c.p;
    a.cd = r->cd_.p;
    a.cwd = r->cwd.p;
    a.cwc = r->cwc.p;
    a.nmv = r->nmv.p;
    a.ncand = r->ncand.p;
    a.tmp_a = r->tmp_a.p;
    a.tmp_b = r->tmp_b.p;
    a.rc_u = r->rc_u.p;
    a.rc_cd = r->rc_cd.p;
    a.rc_vu = r->rc_vu.p;
    a.rc_dw = r->rc_dw.p;
    int ubits = 1;
    while (((int64_t)1 << ubits) < n) ubits++;
    a.ubits = ubits;
    a.max_sweeps = o.max_sweeps;
    a.recheck_from = RECHECK_FROM;
    a.res_p = o.res_p;
    a.res_q = o.res_q;
    a.racy = o.racy > 0 ? 1 : 0;
    if (o.trace) prepare_trace(*r, g, S, s);
    return r;
}

// Returns the number of moves of the phase.
static int64_t finish_move(PhaseRun &r, RunStats &st, cudaStream_t s) {
    int32_t conv = 0;
    std::vector<Counters> per;
    const int32_t runs = read_counters(r, &conv, per, st, s);
    if (r.a.g.n == 0) return 0;   // an empty graph runs no sweep (nothing to decide)
    if (r.cls_ns.p) record_trace(r, runs, s);
    int64_t total = 0;
    for (const Counters &h : per) {
        st.sweeps++;
        st.moves += h.moved;
        st.entries += h.entries;
        st.candidates += h.candidates;
        st.decisions += h.decisions;
        total += h.moved;
        if (r.profile)
            st.k_bytes += 40.0 * h.decisions + (8.0 + wbytes(r.wk)) * h.entries + 8.0 * h.candidates + 12.0 * h.moved;
    }
    if (!conv) st.converged = 0;
    return total;
}

// PLP run on g from the singleton labelling, labels in zeta.
static std::unique_ptr<PhaseRun> prepare_plp(const GraphView &g, const Schedule &S, int32_t *zeta, uint64_t seed,
                                             double theta, const RunOpts &o, cudaStream_t s) {
    auto r = std::make_unique<PhaseRun>();
    r->plp = true;
    r->wk = g.wk;
    r->big = needs_big(g.W);
    r->profile = o.profile;
    r->work = g.nnz + g.n;
    r->quantum = o.team_quantum;
    r->team_min = o.team_min;
    r->listed = S.off[(int64_t)S.ncol * NBINS];
    r->a = phase_args(g, S, zeta);
    r->active.alloc(g.n, s);
    if (g.n) CD_CUDA(cudaMemsetAsync(r->active.p, 1, g.n, s));
    iota32(zeta, g.n, s);
    alloc_counters(*r, o.max_iters + 1, S.nhubs, 0, s);
    r->a.active = r->active.p;
    r->a.seed = seed;
    r->a.theta = theta;
    r->a.max_iters = o.max_iters;
    return r;
}

static void finish_plp(PhaseRun &r, RunStats &st, cudaStream_t s) {
    int32_t conv = 0;
    std::vector<Counters> per;
    const int32_t iters = read_counters(r, &conv, per, st, s);
    for (const Counters &h : per) {
        st.moves += h.moved;
        st.entries += h.entries;
        st.candidates += h.candidates;
        st.decisions += h.decisions;
        if (r.profile)
            st.k_bytes += 5.0 * r.listed + 20.0 * h.decisions + (8.0 + wbytes(r.wk)) * h.entries + 4.0 * h.moved;
    }
    st.iters += iters;
    if (!conv) st.converged = 0;
}

// ---------------------------------------------------------------------------
// Kernels between phases: prolongation and the EPP core (Eq. 2).
// ---------------------------------------------------------------------------
__global__ void k_prolong(int32_t *zeta, const int64_t *rank, const int32_t *up, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        zeta[i] = up[rank[zeta[i]]];
}

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

// ---------------------------------------------------------------------------
// Jobs
// ---------------------------------------------------------------------------
struct Level {
    OwnedGraph own;
    GraphView g;
    Schedule S;
    DBuf<int32_t> zeta;
    DBuf<int64_t> rank;
};

enum Stage {
    ST_START,      // nothing done yet
    ST_PLP_WAIT,   // PLP run launched
    ST_EPP_WAIT,   // EPP base runs launched
    ST_DOWN_WAIT,  // move phase of the deepest level launched
    ST_UP,         // prolong to level `up`
    ST_UP_WAIT,    // refinement move phase of level `up` launched
    ST_PLM_DONE,   // labels of the PLM graph in L[0]->zeta
    ST_FINAL,      // labels in place: modularity, release
};

struct JobState {
    int stage = ST_START;
    Clock::time_point t0;
    GraphView g;                  // graph of the PLM part (input, or EPP's core graph)
    std::vector<std::unique_ptr<Level>> L;
    int up = -1;
    std::unique_ptr<PhaseRun> run;
    // EPP
    std::vector<std::unique_ptr<Schedule>> base_S;
    std::vector<std::unique_ptr<PhaseRun>> base_runs;
    DBuf<int32_t> base, core;
    DBuf<int64_t> core_rank;
    OwnedGraph cg;
    bool epp_plm = false;
};

Job::Job(const JobSpec &s) : spec(s), state(std::make_unique<JobState>()) {}

void Job::release() {
    state.reset();   // stream-ordered frees on `stream`
    if (own_stream) {
        cudaStreamSynchronize(stream);
        cudaStreamDestroy(stream);
        own_stream = false;
    }
    stream = nullptr;
}

Job::~Job() { release(); }

// Level `L.back()`: schedule, singleton labels, move phase.
static void start_level(Job &j, cudaStream_t s) {
    JobState &x = *j.state;
    Level &lv = *x.L.back();
    auto t = Clock::now();
    build_schedule(lv.g, j.spec.o.seed, j.spec.o.bins, lv.S, s, j.spec.o.racy);
    j.st.ms_color += ms_since(t);
    if (x.L.size() == 1 && j.st.colors0 < 0) j.st.colors0 = lv.S.ncol;
    lv.zeta.alloc(lv.g.n, s);
    iota32(lv.zeta.p, lv.g.n, s);
    x.run = prepare_move(lv.g, lv.S, lv.zeta.p, lv.g.vol, j.spec.o, s);
    x.stage = ST_DOWN_WAIT;
}

static void begin_plm(Job &j, cudaStream_t s) {
    JobState &x = *j.state;
    x.L.clear();
    x.L.push_back(std::make_unique<Level>());
    x.L[0]->g = x.g;
    start_level(j, s);
}

// Advances a job until it waits for a launch or is finished.
static void advance_impl(Job &j, cudaStream_t s) {
    JobState &x = *j.state;
    const JobSpec &sp = j.spec;
    RunStats &st = j.st;
    const int64_t n0 = sp.g.n;
    for (;;) {
        switch (x.stage) {
        case ST_START: {
            x.t0 = Clock::now();
            if (sp.algo == ALGO_PLP) {
                x.L.push_back(std::make_unique<Level>());
                Level &lv = *x.L[0];
                lv.g = sp.g;
                auto t = Clock::now();
                build_schedule(sp.g, sp.o.seed, sp.o.bins, lv.S, s);   // PLP keeps the colour classes
                st.ms_color += ms_since(t);
                if (st.colors0 < 0) st.colors0 = lv.S.ncol;
                x.run = prepare_plp(sp.g, lv.S, j.labels(), sp.o.seed, sp.theta, sp.o, s);
                x.stage = ST_PLP_WAIT;
                return;
            }
            if (sp.algo == ALGO_EPP) {
                const int b = sp.ensemble;
                x.base.alloc((size_t)b * n0, s);
                for (int i = 0; i < b; i++) {
                    const uint64_t seed = sp.o.seed + (uint64_t)i;
                    x.base_S.push_back(std::make_unique<Schedule>());
                    auto t = Clock::now();
                    build_schedule(sp.g, seed, sp.o.bins, *x.base_S[i], s);
                    st.ms_color += ms_since(t);
                    if (i == 0) st.colors0 = x.base_S[0]->ncol;
                    x.base_runs.push_back(
                        prepare_plp(sp.g, *x.base_S[i], x.base.p + (size_t)i * n0, seed, sp.theta, sp.o, s));
                }
                x.stage = ST_EPP_WAIT;
                return;
            }
            x.g = sp.g;
            begin_plm(j, s);
            return;
        }
        case ST_PLP_WAIT: {
            finish_plp(*x.run, st, s);
            x.run.reset();
            st.ncomm = (int32_t)compact_labels(j.labels(), n0, s);
            st.levels = 1;
            x.L.clear();
            x.stage = ST_FINAL;
            break;
        }
        case ST_EPP_WAIT: {
            const int b = sp.ensemble;
            for (int i = 0; i < b; i++) {
                finish_plp(*x.base_runs[i], st, s);
                compact_labels(x.base.p + (size_t)i * n0, n0, s);
            }
            x.base_runs.clear();
            x.base_S.clear();
            x.core.alloc(n0, s);
            if (n0) {
                CD_CUDA(cudaMemcpyAsync(x.core.p, x.base.p, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                for (int i = 1; i < b; i++) fold_core(x.core.p, x.base.p + (size_t)i * n0, n0, s);
            }
            x.base.release();
            auto t = Clock::now();
            x.core_rank.alloc(n0, s);
            coarsen_graph(sp.g, x.core.p, x.core_rank.p, x.cg, s, sp.o.scratch_budget);
            x.core_rank.release();
            st.ms_coarsen += ms_since(t);
            x.g = x.cg.view;
            x.epp_plm = true;
            begin_plm(j, s);
            return;
        }
        case ST_DOWN_WAIT: {
            Level &lv = *x.L.back();
            const int64_t moved = finish_move(*x.run, st, s);
            x.run.reset();
            if (moved == 0 || (int)x.L.size() >= sp.o.max_levels) {
                // an empty graph has no level that ran a move phase
                st.levels += lv.g.n > 0 ? (int32_t)x.L.size() : 0;
                st.ncomm = (int32_t)compact_labels(lv.zeta.p, lv.g.n, s);
                x.up = (int)x.L.size() - 2;
                x.stage = ST_UP;
                break;
            }
            if (sp.o.scratch_budget > 0) lv.S = Schedule();   // low-memory mode: rebuilt if a refinement needs it
            auto t = Clock::now();
            lv.rank.alloc(lv.g.n, s);
            auto nx = std::make_unique<Level>();
            coarsen_graph(lv.g, lv.zeta.p, lv.rank.p, nx->own, s, sp.o.scratch_budget);
            st.ms_coarsen += ms_since(t);
            if (sp.o.racy > 0 && nx->own.view.n == lv.g.n) {
                // the racy schedule's moves only exchanged labels (every community
                // is still one vertex): no coarser level, this one is the deepest
                nx.reset();
                lv.rank.release();
                st.levels += (int32_t)x.L.size();
                st.ncomm = (int32_t)compact_labels(lv.zeta.p, lv.g.n, s);
                x.up = (int)x.L.size() - 2;
                x.stage = ST_UP;
                break;
            }
            nx->g = nx->own.view;
            x.L.push_back(std::move(nx));
            start_level(j, s);
            return;
        }
        case ST_UP: {
            if (x.up < 0) {
                x.stage = ST_PLM_DONE;
                break;
            }
            Level &lv = *x.L[x.up];
            const int64_t n = lv.g.n;
            if (n) { k_prolong<<<grid_for(n, kBlock, 152 * 32), kBlock, 0, s>>>(lv.zeta.p, lv.rank.p, x.L[x.up + 1]->zeta.p, n); ::cd::note_launch(); }
            CD_LAUNCH_CHECK();
            x.L.pop_back();
            if (sp.refine) {
                if (lv.S.ncol == 0 && lv.g.n > 0) {
                    // low-memory mode freed this level's schedule: the same
                    // seed colours the level again into the same classes
                    auto t = Clock::now();
                    build_schedule(lv.g, sp.o.seed, sp.o.bins, lv.S, s, sp.o.racy);
                    st.ms_color += ms_since(t);
                }
                x.run = prepare_move(lv.g, lv.S, lv.zeta.p, nullptr, sp.o, s);
                x.stage = ST_UP_WAIT;
                return;
            }
            x.up--;
            break;
        }
        case ST_UP_WAIT: {
            Level &lv = *x.L[x.up];
            finish_move(*x.run, st, s);
            x.run.reset();
            st.ncomm = (int32_t)compact_labels(lv.zeta.p, lv.g.n, s);
            x.up--;
            x.stage = ST_UP;
            break;
        }
        case ST_PLM_DONE: {
            Level &top = *x.L[0];
            if (x.epp_plm) {
                if (n0) { k_gather_core<<<grid_for(n0, kBlock, 152 * 32), kBlock, 0, s>>>(top.zeta.p, x.core.p, n0, j.labels()); ::cd::note_launch(); }
                CD_LAUNCH_CHECK();
                st.ncomm = (int32_t)compact_labels(j.labels(), n0, s);
            } else if (n0) {
                CD_CUDA(cudaMemcpyAsync(j.labels(), top.zeta.p, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            }
            x.L.clear();
            x.stage = ST_FINAL;
            break;
        }
        case ST_FINAL: {
            if (sp.want_mod) j.mod = modularity(sp.g, j.labels(), s);
            CD_CUDA(cudaStreamSynchronize(s));
            st.ms_total += ms_since(x.t0);
            j.done = true;
            return;
        }
        }
    }
}

static std::atomic<int64_t> g_fail_order{0};

static void advance(Job &j) {
    if (j.done) return;
    try {
        advance_impl(j, j.stream);
        // the batched launch (another stream) reads what this step wrote
        CD_CUDA(cudaStreamSynchronize(j.stream));
    } catch (const Error &e) {
        j.status = e.status;
        j.msg = e.msg;
    } catch (const std::bad_alloc &) {
        j.status = CD_ENOMEM;
        j.msg = "host allocation failed";
    }
    if (j.status != CD_OK) {
        j.fail_order = g_fail_order.fetch_add(1);
        j.done = true;
    }
    if (j.done) j.release();
}

// ---------------------------------------------------------------------------
// Host worker threads, each with its own stream.
// ---------------------------------------------------------------------------
class WorkerPool {
  public:
    WorkerPool(int n, int device) : dev_(device) {
        for (int w = 0; w < n; w++) threads_.emplace_back([this]() { loop(); });
    }
    ~WorkerPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    int size() const { return (int)threads_.size(); }
    // fn(i) for i in [0, count); fn must not throw.
    void run(int count, const std::function<void(int)> &fn) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            fn_ = &fn;
            count_ = count;
            next_.store(0);
            pending_ = (int)threads_.size();
            gen_++;
        }
        cv_.notify_all();
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [this]() { return pending_ == 0; });
        fn_ = nullptr;
    }

  private:
    void loop() {
        cudaSetDevice(dev_);
        uint64_t seen = 0;
        for (;;) {
            const std::function<void(int)> *fn;
            int count;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&]() { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                fn = fn_;
                count = count_;
            }
            for (;;) {
                const int i = next_.fetch_add(1);
                if (i >= count) break;
                (*fn)(i);
            }
            std::lock_guard<std::mutex> lk(mu_);
            if (--pending_ == 0) done_cv_.notify_all();
        }
    }
    int dev_;
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)> *fn_ = nullptr;
    std::atomic<int> next_{0};
    int count_ = 0, pending_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
Engine::Engine(cudaStream_t s, int workers) : s_(s) {
    if (workers > 0) {
        int dev = 0;
        CD_CUDA(cudaGetDevice(&dev));
        pool_ = std::make_unique<WorkerPool>(workers, dev);
    }
}

Engine::~Engine() = default;

void Engine::add(Job *j) {
    // labels the job keeps after it finishes live on the engine's stream
    if (!j->spec.labels) {
        j->own_labels.alloc(j->spec.g.n, s_);
        CD_CUDA(cudaStreamSynchronize(s_));
    }
    if (pool_) {
        CD_CUDA(cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking));
        j->own_stream = true;
    } else {
        j->stream = s_;
    }
    active_.push_back(j);
}

void Engine::step() {
    std::vector<Job *> act = active_;
    if (pool_ && act.size() > 1) {
        pool_->run((int)act.size(), [&](int i) { advance(*act[i]); });
    } else {
        for (Job *j : act) advance(*j);
    }
    std::vector<PhaseRun *> runs;
    for (Job *j : act) {
        if (j->done) continue;
        JobState &x = *j->state;
        if (x.run) runs.push_back(x.run.get());
        for (auto &r : x.base_runs) runs.push_back(r.get());
    }
    if (!runs.empty()) launch(runs);
    active_.erase(std::remove_if(active_.begin(), active_.end(), [](Job *j) { return j->done; }), active_.end());
}

// Tiers of one launch: runs with the same smallest useful team size share a
// tier; tiers get blocks in proportion to their work.
struct LaunchPlan {
    BatchArgs b{};
    int grid = 0, nteams = 0;
    std::vector<PhaseRun *> order;   // runs in tier order
};

static LaunchPlan plan_launch(std::vector<PhaseRun *> runs, int G) {
    int64_t quantum = runs[0]->quantum;
    int team_min = runs[0]->team_min;
    for (const PhaseRun *r : runs) {
        quantum = std::min(quantum, r->quantum);
        team_min = std::max(team_min, r->team_min);
    }
    quantum = std::max<int64_t>(quantum, 1);
    team_min = std::max(team_min, 1);
    auto need = [&](const PhaseRun *r) {
        const int64_t q = (r->work + quantum - 1) / quantum;
        int t = 1;
        while (t < q && t < G) t <<= 1;
        return std::min(t, G);
    };
    std::stable_sort(runs.begin(), runs.end(), [&](const PhaseRun *x, const PhaseRun *y) {
        const int nx = need(x), ny = need(y);
        return nx != ny ? nx > ny : x->work > y->work;
    });
    struct T { int need, count = 0, blocks = 0, first = 0; double work = 0; };
    std::vector<T> tiers;
    for (int i = 0; i < (int)runs.size(); i++) {
        const int nd = need(runs[i]);
        if (tiers.empty() || tiers.back().need != nd) {
            if ((int)tiers.size() == MAX_TIERS) {
                // merge into the last tier (cannot happen for power-of-two sizes <= 2048)
                tiers.back().count++;
                tiers.back().work += (double)runs[i]->work + 1;
                continue;
            }
            tiers.push_back(T{nd, 0, 0, i, 0});
        }
        tiers.back().count++;
        tiers.back().work += (double)runs[i]->work + 1;
    }
    double W = 0;
    for (auto &t : tiers) W += t.work;
    int total = 0;
    for (auto &t : tiers) {
        t.blocks = std::max(1, (int)std::floor(G * t.work / W));
        total += t.blocks;
    }
    while (total > G) {
        int j = 0;
        for (int i = 1; i < (int)tiers.size(); i++) if (tiers[i].blocks > tiers[j].blocks) j = i;
        tiers[j].blocks--;
        total--;
    }
    while (total < G) {
        int j = 0;
        for (int i = 1; i < (int)tiers.size(); i++)
            if (tiers[i].work / tiers[i].blocks > tiers[j].work / tiers[j].blocks) j = i;
        tiers[j].blocks++;
        total++;
    }
    LaunchPlan p;
    p.order = runs;
    p.b.ntiers = (int32_t)tiers.size();
    int begin = 0, team0 = 0;
    for (int i = 0; i < (int)tiers.size(); i++) {
        const T &t = tiers[i];
        int ts = std::min(t.need, std::max(1, t.blocks / std::min(t.count, team_min)));
        if ((int64_t)t.count * ts < t.blocks) ts = t.blocks / t.count;
        const int teams = std::max(1, t.blocks / ts);
        Tier &d = p.b.tiers[i];
        d.begin = begin;
        d.blocks = teams * ts;
        d.team_size = ts;
        d.team0 = team0;
        d.first = t.first;
        d.count = t.count;
        begin += d.blocks;
        team0 += teams;
    }
    p.grid = begin;
    p.nteams = team0;
    return p;
}

// The planner on bare phase sizes (host only; no device work): one run per
// entry of `work`, every run with the same launch shape.
PlanView plan_for_sizes(const std::vector<int64_t> &work, int64_t quantum, int32_t team_min, int grid_max) {
    std::vector<std::unique_ptr<PhaseRun>> own;
    std::vector<PhaseRun *> runs;
    for (int64_t wk : work) {
        own.push_back(std::make_unique<PhaseRun>());
        own.back()->work = wk;
        own.back()->quantum = quantum;
        own.back()->team_min = team_min;
        runs.push_back(own.back().get());
    }
    const LaunchPlan lp = plan_launch(runs, grid_max);
    PlanView v;
    v.grid = lp.grid;
    v.nteams = lp.nteams;
    for (int i = 0; i < lp.b.ntiers; i++) {
        const Tier &t = lp.b.tiers[i];
        v.tiers.push_back(PlanTier{t.begin, t.blocks, t.team_size, t.team0, t.first, t.count});
    }
    for (const PhaseRun *r : lp.order)
        for (size_t k = 0; k < runs.size(); k++)
            if (runs[k] == r) v.order.push_back((int32_t)k);
    return v;
}

void Engine::launch(std::vector<PhaseRun *> &runs) {
    const auto t = Clock::now();
    // group by kernel instantiation, keeping the order of first appearance
    std::vector<std::vector<PhaseRun *>> groups;
    auto key = [](const PhaseRun *r) { return (r->plp ? 8 : 0) + r->wk * 2 + (r->big ? 1 : 0); };
    for (PhaseRun *r : runs) {
        bool placed = false;
        for (auto &g : groups)
            if (key(g[0]) == key(r)) { g.push_back(r); placed = true; break; }
        if (!placed) groups.push_back({r});
    }
    struct Issued {
        LaunchPlan plan;
        DBuf<PhaseArgs> args;
        DBuf<GridBarrier> bars;
        DBuf<unsigned int> queues;
        DBuf<int32_t> team_graph;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Issued() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    };
    std::vector<std::unique_ptr<Issued>> issued;
    try {
        for (auto &g : groups) {
            const void *kern = g[0]->plp ? plp_batch_kernel(g[0]->wk, g[0]->big) : move_batch_kernel(g[0]->wk, g[0]->big);
            int G = persistent_grid(kern);
            if (share_ < 1.0) G = std::max(1, (int)(G * share_));
            ensure_block_tables(G);
            auto is = std::make_unique<Issued>();
            is->plan = plan_launch(g, G);
            LaunchPlan &p = is->plan;
            p.b.gt_keys = gt_keys_.p;
            p.b.gt_vals = gt_vals_.p;
            std::vector<PhaseArgs> host(p.order.size());
            for (size_t i = 0; i < p.order.size(); i++) host[i] = p.order[i]->a;
            is->args.alloc(host.size(), s_);
            CD_CUDA(cudaMemcpyAsync(is->args.p, host.data(), host.size() * sizeof(PhaseArgs), cudaMemcpyHostToDevice, s_));
            is->bars.alloc(p.nteams, s_);
            is->bars.zero();
            is->queues.alloc(p.b.ntiers, s_);
            is->queues.zero();
            is->team_graph.alloc(p.nteams, s_);
            p.b.graphs = is->args.p;
            p.b.bars = is->bars.p;
            p.b.queues = is->queues.p;
            p.b.team_graph = is->team_graph.p;
            bool prof = false;
            for (PhaseRun *r : g) prof = prof || r->profile;
            if (prof) {
                CD_CUDA(cudaEventCreate(&is->e0));
                CD_CUDA(cudaEventCreate(&is->e1));
                CD_CUDA(cudaEventRecord(is->e0, s_));
            }
            {
                Residency res(kern, p.grid, PHASE_SMEM);
                launch_batch(kern, p.b, p.grid, s_);
                if (prof) CD_CUDA(cudaEventRecord(is->e1, s_));
                CD_CUDA(cudaStreamSynchronize(s_));
            }
            issued.push_back(std::move(is));
            launches++;
        }
        CD_CUDA(cudaStreamSynchronize(s_));
        const double wall = ms_since(t);
        for (auto &is : issued) {
            std::vector<GridBarrier> hb(is->plan.nteams);
            CD_CUDA(cudaMemcpyAsync(hb.data(), is->bars.p, hb.size() * sizeof(GridBarrier), cudaMemcpyDeviceToHost, s_));
            CD_CUDA(cudaStreamSynchronize(s_));
            bool timeout = false;
            for (const GridBarrier &b : hb) timeout = timeout || b.err != 0;
            float ms = 0;
            if (is->e0) CD_CUDA(cudaEventElapsedTime(&ms, is->e0, is->e1));
            for (PhaseRun *r : is->plan.order) {
                r->wall_ms = wall;
                r->launch_ms = ms;
                if (timeout) {
                    r->fail = CD_ETIMEOUT;
                    r->fail_msg = "a team barrier of the persistent kernel timed out";
                }
            }
        }
    } catch (const Error &e) {
        for (PhaseRun *r : runs) {
            r->fail = e.status;
            r->fail_msg = e.msg;
        }
        cudaStreamSynchronize(s_);
        gt_blocks_ = 0;   // a failed launch may have left entries behind: clear before the next one
    }
}

// Role-3b tables, GT_SLOTS per block of the largest grid: all keys -1 and
// values 0, which every use restores.
void Engine::ensure_block_tables(int blocks) {
    if (blocks <= gt_blocks_) return;
    const size_t slots = (size_t)blocks * GT_SLOTS;
    gt_keys_.alloc(slots, s_);
    gt_vals_.alloc(slots, s_);
    CD_CUDA(cudaMemsetAsync(gt_keys_.p, 0xff, slots * sizeof(int32_t), s_));
    gt_vals_.zero();
    gt_blocks_ = blocks;
}

void run_jobs(std::vector<Job *> &jobs, cudaStream_t s, int workers) {
    Engine e(s, (int)jobs.size() > 1 ? workers : 0);
    for (Job *j : jobs) e.add(j);
    while (e.busy()) e.step();
    const Job *first = nullptr;
    for (const Job *j : jobs)
        if (j->status != CD_OK && (!first || j->fail_order < first->fail_order)) first = j;
    if (first) raise(first->status, "%s", first->msg.c_str());
}

static void run_single(JobSpec sp, RunStats &st, cudaStream_t s) {
    Job j(sp);
    std::vector<Job *> v{&j};
    run_jobs(v, s, 0);
    st = j.st;
}

void run_plm(const GraphView &g, bool refine, const RunOpts &o, int32_t *labels, RunStats &st, cudaStream_t s) {
    JobSpec sp;
    sp.g = g;
    sp.algo = ALGO_PLM;
    sp.refine = refine;
    sp.o = o;
    sp.labels = labels;
    run_single(sp, st, s);
}

void run_plp(const GraphView &g, const RunOpts &o, double theta, int32_t *labels, RunStats &st, cudaStream_t s) {
    JobSpec sp;
    sp.g = g;
    sp.algo = ALGO_PLP;
    sp.theta = theta;
    sp.o = o;
    sp.labels = labels;
    run_single(sp, st, s);
}

void run_epp(const GraphView &g, int b, bool final_refine, const RunOpts &o, double theta, int32_t *labels,
             RunStats &st, cudaStream_t s) {
    JobSpec sp;
    sp.g = g;
    sp.algo = ALGO_EPP;
    sp.ensemble = b;
    sp.refine = final_refine;
    sp.theta = theta;
    sp.o = o;
    sp.labels = labels;
    run_single(sp, st, s);
}

// EPP(b, Base, Final) with iterated ensembles.  Round r runs b base jobs
// (seeds seed + r b + i) on the current graph in one batch, folds their exact
// core communities (Eq. 2), and coarsens by them; a round after the first
// is taken only if its core merges vertices and has strictly higher
// modularity than the previous round's.  The final PLM / PLMR job runs on
// the last core graph and its labels are prolonged through every round.
void run_epp_general(const GraphView &g, int b, int base, bool final_refine, int rounds, const RunOpts &o,
                     double theta, int32_t *labels, RunStats &st, cudaStream_t s) {
    if (base == EPP_BASE_PLP && rounds == 1) {   // Algorithm 5 as one job: the bases share one launch
        run_epp(g, b, final_refine, o, theta, labels, st, s);
        st.levels = 1;                            // one core graph taken
        return;
    }
    struct Round {
        OwnedGraph cg;
        DBuf<int32_t> core;    // core community of each vertex of the round's input graph
        DBuf<int64_t> rank;    // core label -> vertex of cg
    };
    std::vector<std::unique_ptr<Round>> taken;
    GraphView cur = g;
    double prev = 0.0;
    int64_t base_iters = 0;
    const int hw = (int)std::thread::hardware_concurrency();
    const int workers = std::max(1, std::min({16, b, hw > 0 ? hw : 4}));
    for (int r = 0; r < rounds; r++) {
        const int64_t nc = cur.n;
        DBuf<int32_t> bl((size_t)b * nc, s);
        std::vector<std::unique_ptr<Job>> jobs;
        std::vector<Job *> jp;
        for (int i = 0; i < b; i++) {
            JobSpec sp;
            sp.g = cur;
            sp.algo = base == EPP_BASE_PLP ? ALGO_PLP : ALGO_PLM;
            sp.refine = base == EPP_BASE_PLMR;
            sp.theta = theta;
            sp.o = o;
            sp.o.seed = o.seed + (uint64_t)r * (uint64_t)b + (uint64_t)i;
            sp.labels = bl.p + (size_t)i * nc;
            jobs.push_back(std::make_unique<Job>(sp));
            jp.push_back(jobs.back().get());
        }
        if (nc > 0) run_jobs(jp, s, workers);
        for (const auto &j : jobs) base_iters += j->st.iters;
        auto rd = std::make_unique<Round>();
        rd->core.alloc(nc, s);
        if (nc) {
            CD_CUDA(cudaMemcpyAsync(rd->core.p, bl.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            for (int i = 1; i < b; i++) fold_core(rd->core.p, bl.p + (size_t)i * nc, nc, s);
        }
        const int64_t k = nc ? compact_labels(rd->core.p, nc, s) : 0;
        const double q = modularity(cur, rd->core.p, s);
        if (r > 0 && (k == nc || q <= prev)) break;     // no contraction or no gain
        prev = q;
        rd->rank.alloc(nc, s);
        coarsen_graph(cur, rd->core.p, rd->rank.p, rd->cg, s, o.scratch_budget);
        cur = rd->cg.view;
        taken.push_back(std::move(rd));
    }
    DBuf<int32_t> zf(cur.n, s);
    RunStats fs;
    run_plm(cur, final_refine, o, zf.p, fs, s);
    // prolong through the rounds, deepest first: core <- final labels of its
    // coarse vertex (k_prolong, in place)
    const int32_t *up = zf.p;
    for (int l = (int)taken.size() - 1; l >= 0; l--) {
        Round &rd = *taken[l];
        const int64_t nl = l == 0 ? g.n : taken[l - 1]->cg.view.n;
        if (nl) { k_prolong<<<grid_for(nl, kBlock, 152 * 32), kBlock, 0, s>>>(rd.core.p, rd.rank.p, up, nl); ::cd::note_launch(); }
        CD_LAUNCH_CHECK();
        up = rd.core.p;
    }
    if (g.n) CD_CUDA(cudaMemcpyAsync(labels, up, g.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    const int64_t k = g.n ? compact_labels(labels, g.n, s) : 0;
    CD_CUDA(cudaStreamSynchronize(s));
    st = fs;
    st.iters += base_iters;
    st.levels = (int32_t)taken.size();
    st.ncomm = (int32_t)k;
}

}  // namespace cd
