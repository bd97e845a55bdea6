// PLP decide kernels (Algorithm 1).
#include "move_dispatch.cuh"

namespace cd {

template <>
void decide_class<true>(int wk, bool big, const SweepCtx &c, const ClassBins &cb, cudaStream_t s, LaunchTimer &t) {
    if (!big) {
        if (wk == W_UNIT) decide_class_t<W_UNIT, false, true>(c, cb, s, t);
        else if (wk == W_I32) decide_class_t<W_I32, false, true>(c, cb, s, t);
        else raise(CD_ECUDA, "int64 weights need the 128-bit path");
    } else {
        if (wk == W_UNIT) decide_class_t<W_UNIT, true, true>(c, cb, s, t);
        else if (wk == W_I32) decide_class_t<W_I32, true, true>(c, cb, s, t);
        else decide_class_t<W_I64, true, true>(c, cb, s, t);
    }
}

}  // namespace cd
