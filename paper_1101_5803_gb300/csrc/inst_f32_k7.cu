// float kernels, 7x7 PSF
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_k7(KernelTable& t) {
    t.cgls[0][0][7] = (const void*)k_cgls<float, 7, false>;
    t.cgls[0][1][7] = (const void*)k_cgls<float, 7, true>;

}
}  // namespace mirage
