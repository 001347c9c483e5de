// double kernels (FP64 mode)
#include "kernels.cuh"
#include "table.h"

namespace mirage {
void fill_f64(KernelTable& t) {
    t.cgls[1][0][5] = (const void*)k_cgls<double, 5, PLACE_SMEM>;
    t.cgls[1][0][0] = (const void*)k_cgls<double, 0, PLACE_SMEM>;
    t.cgls[1][1][0] = (const void*)k_cgls<double, 0, PLACE_GLOBAL>;
    t.fwd[1][0] = (const void*)k_forward<double, 0>;
    t.raytrace[1] = (const void*)k_raytrace<double>;
    t.rt_trace[1] = (const void*)k_rt_trace<double>;
    t.rt_place[1] = (const void*)k_rt_place<double>;
    t.rt_scatter[1] = (const void*)k_rt_scatter<double>;
    t.rt_sortcells[1] = (const void*)k_rt_sortcells<double>;
    t.finalize[1] = (const void*)k_finalize<double>;
    t.psf_spectra[1] = (const void*)k_psf_spectra<double>;
}
}  // namespace mirage
