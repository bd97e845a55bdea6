// Launch of the decide kernels of one colour class (instantiated per
// weight kind / gain width in move_plm.cu and move_plp.cu).
#pragma once
#include "move_kernels.cuh"

namespace cd {

struct ClassBins {
    const int32_t *order;      // class vertices, bin by bin (device)
    int64_t off[NBINS + 1];    // bin offsets relative to `order` (host)
    int32_t nb1 = 0, nb2 = 0;  // hub H1 / H2 block counts
};

template <int WK, bool BIG, bool PLP>
void decide_class_t(const SweepCtx &c, const ClassBins &cb, cudaStream_t s, LaunchTimer &t) {
    const int64_t n0 = cb.off[1] - cb.off[0], n1 = cb.off[2] - cb.off[1], n2 = cb.off[3] - cb.off[2];
    const int64_t n3 = cb.off[4] - cb.off[3];
    if (n0) {
        t.before(s);
        { k_decide_group<4, 4, WK, BIG, PLP><<<grid_for(n0, kBlock / 4), kBlock, 0, s>>>(c, cb.order + cb.off[0], n0); ::cd::note_launch(); }
        t.after(s);
    }
    if (n1) {
        t.before(s);
        { k_decide_group<8, 16, WK, BIG, PLP><<<grid_for(n1, kBlock / 8), kBlock, 0, s>>>(c, cb.order + cb.off[1], n1); ::cd::note_launch(); }
        t.after(s);
    }
    if (n2) {
        t.before(s);
        { k_decide_group<32, 128, WK, BIG, PLP><<<grid_for(n2, kBlock / 32), kBlock, 0, s>>>(c, cb.order + cb.off[2], n2); ::cd::note_launch(); }
        t.after(s);
    }
    if (n3) {
        t.before(s);
        { k_decide_block<WK, BIG, PLP><<<grid_for(n3, 1, 152 * 8), kBlock, 0, s>>>(c, cb.order + cb.off[3], n3); ::cd::note_launch(); }
        t.after(s);
    }
    if (cb.nb1) {
        t.before(s);
        { k_hub_aggregate<WK, BIG, PLP><<<cb.nb1, kBlock, 0, s>>>(c); ::cd::note_launch(); }
        { k_hub_decide<WK, BIG, PLP><<<cb.nb2, kBlock, 0, s>>>(c); ::cd::note_launch(); }
        t.after(s);
    }
    CD_LAUNCH_CHECK();
}

template <bool PLP>
void decide_class(int wk, bool big, const SweepCtx &c, const ClassBins &cb, cudaStream_t s, LaunchTimer &t);

// Late-sweep sequential re-check of one class (move_plm.cu).
struct RecheckArgs {
    const int32_t *cu, *cc, *cd;
    const int64_t *cwd, *cwc;
    const unsigned long long *ncand;
    int32_t *zeta;
    const int64_t *vol;
    int64_t *volc;
    int64_t twoW;
    uint64_t *tmp_a, *tmp_b;   // class-sized scratch for long candidate lists
    int ubits;                 // bits of the largest vertex id
    Counters *cnt;
};
void recheck_class(bool big, const RecheckArgs &a, cudaStream_t s);

}  // namespace cd
