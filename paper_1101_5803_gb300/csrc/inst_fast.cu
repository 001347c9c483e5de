// fast-path CGLS kernels (two CTAs per SM; FP32 contexts, images up to 64x64)
#include "fast.cuh"
#include "table.h"

namespace mirage {
void fill_fast(KernelTable& t) {
    t.fast[5][0] = (const void*)k_cgls_fast<5, 4>;
    t.fast[7][0] = (const void*)k_cgls_fast<7, 4>;
    t.fast[9][0] = (const void*)k_cgls_fast<9, 4>;
    t.fast[9][1] = (const void*)k_cgls_fast<9, 9>;
    t.fast[11][0] = (const void*)k_cgls_fast<11, 4>;
    t.fast[11][1] = (const void*)k_cgls_fast<11, 9>;
}
}  // namespace mirage
