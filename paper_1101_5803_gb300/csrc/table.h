// Registry of the compiled kernel instantiations (filled by the inst_*.cu
// translation units, which are compiled in parallel).
#pragma once

namespace mirage {

constexpr int MAX_K = 32;  // tap sides 1..31 (odd); index 0 = runtime-K kernel

struct KernelTable {
    // cgls[prec][place][K], prec 0 = float, 1 = double; place = PLACE_SMEM,
    // PLACE_GLOBAL, PLACE_MID; nullptr = not compiled
    const void* cgls[2][5][MAX_K];
    const void* fwd[2][MAX_K];
    const void* raytrace[2];
    const void* rt_trace[2];  // split ray trace: trace and count (many CTAs per candidate)
    const void* rt_place[2];  //                  scan and place (one CTA per candidate)
    const void* rt_scatter[2];    // parallel placement, one ray per pixel
    const void* rt_sortcells[2];
    const void* finalize[2];
    // fast[K][v][mode]: two-CTA-per-SM FP32 kernel, v = 0 for ns <= 1024,
    // 1 for ns <= 2304; mode = tap source (0 shared, 1 params FFMA, 2 params
    // FFMA2, 3 params FFMA with TF32-rounded factors)
    const void* fast[MAX_K][2][4];
    // iter[prec][K]: fixed-iteration CGLS with the iteration L-curve
    const void* iter[2][MAX_K];
    // fwdb[K]: banded FP32 forward batch (one ray per pixel)
    const void* fwdb[MAX_K];
    const void* pixmap;  // pixel-ordered ray map for the banded forward batch
    const void* psf_spectra[2];  // PSF spectra of the FFT-convolution problems
};

void fill_f32_k5(KernelTable& t);
void fill_f32_k7(KernelTable& t);
void fill_f32_k9(KernelTable& t);
void fill_f32_k11(KernelTable& t);
void fill_f32_k15(KernelTable& t);
void fill_f32_k21(KernelTable& t);
void fill_f32_gen(KernelTable& t);
void fill_f64(KernelTable& t);
void fill_fast(KernelTable& t);
void fill_iter(KernelTable& t);
void fill_fwd_band(KernelTable& t);

}  // namespace mirage
