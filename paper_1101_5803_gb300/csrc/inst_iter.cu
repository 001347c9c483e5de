// fixed-iteration CGLS with the iteration L-curve and the MC degrees of
// freedom.  The iteration computes in FP64; FP32 contexts keep their FP32
// padded layout (a wider x offset), so they take the runtime-K kernel, which
// reads the offset from the geometry.
#include "iterlc.cuh"
#include "table.h"

namespace mirage {
void fill_iter(KernelTable& t) {
    t.iter[0][0] = (const void*)k_cgls_iter<float, 0>;
    t.iter[1][0] = (const void*)k_cgls_iter<double, 0>;
    t.iter[1][5] = (const void*)k_cgls_iter<double, 5>;
}
}  // namespace mirage
