// float kernels, 5x5 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k5(KernelTable& t) {
    t.cgls[0][0][5] = (const void*)k_cgls<float, 5, PLACE_SMEM>;


}
}  // namespace mirage
