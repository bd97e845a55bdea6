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
