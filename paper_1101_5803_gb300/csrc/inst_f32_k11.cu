// float kernels, 11x11 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k11(KernelTable& t) {
    t.cgls[0][0][11] = (const void*)k_cgls<float, 11, false>;
    t.cgls[0][1][11] = (const void*)k_cgls<float, 11, true>;

}
}  // namespace mirage
