// PLM / PLMR move phase (Algorithm 2): persistent kernel instantiations.
#include "move_dispatch.cuh"

namespace cd {

void launch_move_phase(int wk, bool big, const PhaseArgs &a, cudaStream_t s) {
    if (!big) {
        if (wk == W_UNIT) launch_persistent((const void *)k_move_phase<W_UNIT, false>, a, s);
        else if (wk == W_I32) launch_persistent((const void *)k_move_phase<W_I32, false>, a, s);
        else raise(CD_ECUDA, "int64 weights need the 128-bit gain path");
    } else {
        if (wk == W_UNIT) launch_persistent((const void *)k_move_phase<W_UNIT, true>, a, s);
        else if (wk == W_I32) launch_persistent((const void *)k_move_phase<W_I32, true>, a, s);
        else launch_persistent((const void *)k_move_phase<W_I64, true>, a, s);
    }
}

}  // namespace cd
