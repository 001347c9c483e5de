// float kernels: runtime-K fallbacks, forward batch, ray trace, finalize
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f32_gen(KernelTable& t) {
    t.cgls[0][0][0] = (const void*)k_cgls<float, 0, PLACE_SMEM>;
    t.cgls[0][1][0] = (const void*)k_cgls<float, 0, PLACE_GLOBAL>;
    t.cgls[0][PLACE_GLOBAL2][0] = (const void*)k_cgls<float, 0, PLACE_GLOBAL, 2>;
    t.cgls[0][2][0] = (const void*)k_cgls<float, 0, PLACE_MID>;
    t.cgls[0][PLACE_MID2][0] = (const void*)k_cgls<float, 0, PLACE_MID, 2>;
    t.fwd[0][0] = (const void*)k_forward<float, 0>;
    t.fwd[0][9] = (const void*)k_forward<float, 9>;
    t.raytrace[0] = (const void*)k_raytrace<float>;
    t.rt_trace[0] = (const void*)k_rt_trace<float>;
    t.rt_place[0] = (const void*)k_rt_place<float>;
    t.rt_scatter[0] = (const void*)k_rt_scatter<float>;
    t.rt_sortcells[0] = (const void*)k_rt_sortcells<float>;
    t.finalize[0] = (const void*)k_finalize<float>;
    t.psf_spectra[0] = (const void*)k_psf_spectra<float>;
}
}  // namespace mirage
