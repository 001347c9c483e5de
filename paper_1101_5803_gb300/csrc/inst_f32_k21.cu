// float kernels, 21x21 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k21(KernelTable& t) {
    t.cgls[0][0][21] = (const void*)k_cgls<float, 21, PLACE_SMEM>;
    t.cgls[0][1][21] = (const void*)k_cgls<float, 21, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][21] = (const void*)k_cgls<float, 21, PLACE_GLOBAL, 2>;
    t.fwd[0][21] = (const void*)k_forward<float, 21>;
}
}  // namespace mirage
