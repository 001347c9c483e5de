// float kernels, 15x15 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k15(KernelTable& t) {
    t.cgls[0][0][15] = (const void*)k_cgls<float, 15, PLACE_SMEM>;
    t.cgls[0][1][15] = (const void*)k_cgls<float, 15, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][15] = (const void*)k_cgls<float, 15, PLACE_GLOBAL, 2>;
    t.cgls[0][2][15] = (const void*)k_cgls<float, 15, PLACE_MID>;
    t.cgls[0][PLACE_MID2][15] = (const void*)k_cgls<float, 15, PLACE_MID, 2>;

}
}  // namespace mirage
