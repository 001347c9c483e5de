// float kernels, 11x11 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k11(KernelTable& t) {
    t.cgls[0][0][11] = (const void*)k_cgls<float, 11, PLACE_SMEM>;
    t.cgls[0][1][11] = (const void*)k_cgls<float, 11, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][11] = (const void*)k_cgls<float, 11, PLACE_GLOBAL, 2>;
    t.cgls[0][2][11] = (const void*)k_cgls<float, 11, PLACE_MID>;
    t.cgls[0][PLACE_MID2][11] = (const void*)k_cgls<float, 11, PLACE_MID, 2>;

}
}  // namespace mirage
