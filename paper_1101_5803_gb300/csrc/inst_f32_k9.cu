// float kernels, 9x9 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k9(KernelTable& t) {
    t.cgls[0][0][9] = (const void*)k_cgls<float, 9, false>;
    t.cgls[0][1][9] = (const void*)k_cgls<float, 9, true>;
}
}  // namespace mirage
