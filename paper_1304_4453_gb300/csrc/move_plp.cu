// PLP (Algorithm 1): persistent kernel instantiations.
#include "move_dispatch.cuh"

namespace cd {

void launch_plp_run(int wk, bool big, const PhaseArgs &a, cudaStream_t s) {
    if (!big) {
        if (wk == W_UNIT) launch_persistent((const void *)k_plp_run<W_UNIT, false>, a, s);
        else if (wk == W_I32) launch_persistent((const void *)k_plp_run<W_I32, false>, a, s);
        else raise(CD_ECUDA, "int64 weights need the 128-bit path");
    } else {
        if (wk == W_UNIT) launch_persistent((const void *)k_plp_run<W_UNIT, true>, a, s);
        else if (wk == W_I32) launch_persistent((const void *)k_plp_run<W_I32, true>, a, s);
        else launch_persistent((const void *)k_plp_run<W_I64, true>, a, s);
    }
}

}  // namespace cd
