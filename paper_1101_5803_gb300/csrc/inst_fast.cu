// fast-path CGLS kernels (two CTAs per SM; FP32 contexts, images up to 64x64)
//   fast[K][0][mode] (at most 1024 source pixels: four per thread);
//   mode 0 = taps from shared memory (any batch), 1/2 = taps as kernel
//   parameters (one PSF per launch) with FFMA / packed FFMA2
#include "fast.cuh"
#include "table.h"

namespace mirage {
void fill_fast(KernelTable& t) {
    t.fast[5][0][0] = (const void*)k_cgls_fast<5, 4, TAPS_SMEM_X2>;
    t.fast[7][0][0] = (const void*)k_cgls_fast<7, 4, TAPS_SMEM_X2>;
    t.fast[9][0][0] = (const void*)k_cgls_fast<9, 4, TAPS_SMEM_X2>;
    t.fast[11][0][0] = (const void*)k_cgls_fast<11, 4, TAPS_SMEM_X2>;
    t.fast[9][0][1] = (const void*)k_cgls_fast<9, 4, TAPS_PARAM>;
    t.fast[9][0][2] = (const void*)k_cgls_fast<9, 4, TAPS_PARAM_X2>;
    t.fast[9][0][3] = (const void*)k_cgls_fast<9, 4, TAPS_PARAM_TF32>;
    t.fast[5][0][2] = (const void*)k_cgls_fast<5, 4, TAPS_PARAM_X2>;
    t.fast[7][0][2] = (const void*)k_cgls_fast<7, 4, TAPS_PARAM_X2>;
    t.fast[11][0][2] = (const void*)k_cgls_fast<11, 4, TAPS_PARAM_X2>;
}
}  // namespace mirage
