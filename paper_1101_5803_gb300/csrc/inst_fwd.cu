// banded forward-batch kernels (FP32, one ray per pixel, taps as parameters)
#include "forward.cuh"
#include "table.h"

namespace mirage {
void fill_fwd_band(KernelTable& t) {
    t.fwdb[9] = (const void*)k_forward_band<9>;
    t.fwdb[11] = (const void*)k_forward_band<11>;
    t.fwdb[15] = (const void*)k_forward_band<15>;
    t.fwdb[21] = (const void*)k_forward_band<21>;
    t.pixmap = (const void*)k_pixmap<0>;
}
}  // namespace mirage
