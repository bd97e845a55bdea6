// PLP (Algorithm 1): persistent batch kernel instantiations.
#include "move_dispatch.cuh"

namespace cd {

const void *plp_batch_kernel(int wk, bool big) {
    if (!big) {
        if (wk == W_UNIT) return (const void *)k_plp_batch<W_UNIT, false>;
        if (wk == W_I32) return (const void *)k_plp_batch<W_I32, false>;
        raise(CD_ECUDA, "int64 weights need the 128-bit path");
    }
    if (wk == W_UNIT) return (const void *)k_plp_batch<W_UNIT, true>;
    if (wk == W_I32) return (const void *)k_plp_batch<W_I32, true>;
    return (const void *)k_plp_batch<W_I64, true>;
}

}  // namespace cd
