// float kernels, 9x9 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k9(KernelTable& t) {
    t.cgls[0][0][9] = (const void*)k_cgls<float, 9, PLACE_SMEM>;
    t.cgls[0][1][9] = (const void*)k_cgls<float, 9, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][9] = (const void*)k_cgls<float, 9, PLACE_GLOBAL, 2>;
    t.cgls[0][2][9] = (const void*)k_cgls<float, 9, PLACE_MID>;
    t.cgls[0][PLACE_MID2][9] = (const void*)k_cgls<float, 9, PLACE_MID, 2>;
}
}  // namespace mirage
