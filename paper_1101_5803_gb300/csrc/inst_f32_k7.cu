// float kernels, 7x7 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k7(KernelTable& t) {
    t.cgls[0][0][7] = (const void*)k_cgls<float, 7, PLACE_SMEM>;
    t.cgls[0][1][7] = (const void*)k_cgls<float, 7, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][7] = (const void*)k_cgls<float, 7, PLACE_GLOBAL, 2>;
    t.cgls[0][2][7] = (const void*)k_cgls<float, 7, PLACE_MID>;
    t.cgls[0][PLACE_MID2][7] = (const void*)k_cgls<float, 7, PLACE_MID, 2>;

}
}  // namespace mirage
