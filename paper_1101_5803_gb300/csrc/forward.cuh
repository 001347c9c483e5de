// Banded forward batch (FP32 contexts, one ray per pixel): model = B L s and
// Eq. chi2 for many sources at one lens (Section 3.2's refinement fitness).
//
// One CTA of FWD_THREADS threads per source at a time (persistent over the
// sources).  The source vector is staged in shared memory; the image is
// processed in bands of whole tile rows, each band's zero-padded L s values
// (its rows plus the K-1 halo rows) gathered straight into shared memory
// through the ray trace's pixel -> ray index, so L s never goes to global
// memory.  Each thread owns one 4x4 tile of the band and convolves it with
// the PSF taps held as kernel parameters (read by FFMA from the constant
// bank); chi^2 is accumulated in FP64.
#pragma once

#include "fast.cuh"

namespace mirage {

constexpr int FWD_THREADS = 512;
constexpr int MAX_FTAP = 31 * 31;

struct FwdArgs {
    const Prob<float>* probs;
    CandScratch<float> cs;
    const float* S;   // [n_src][ns]
    int n_src;
    float* model;     // nullable [n_src][npix]
    double* chi2;     // [n_src]
    int* status;      // nullable [1]
    int band_tiles;   // tile rows per band
    float ptap[MAX_FTAP];  // flipped PSF (B), row-major K x K
};

// shared memory: source vector, then the band (band rows + K - 1) x Wp
__host__ inline size_t fwd_band_smem(const Prob<float>& P, int band_tiles) {
    return 16 + 2 * 33 * sizeof(double) + align_up<float>(sizeof(float) * P.ns, 16) +
           sizeof(float) * (size_t)(band_tiles * TILE + P.K - 1) * P.Wp;
}

template <int K>
__global__ void __launch_bounds__(FWD_THREADS, 1) k_forward_band(const __grid_constant__ FwdArgs FA) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob<float>& P = FA.probs[0];
    const CandScratch<float>& cs = FA.cs;
    const Geo<float> g = geo_of(P, cs.nent[0]);
    double* red = reinterpret_cast<double*>(smem + 16);
    float* s_sh = reinterpret_cast<float*>(smem + 16 + 2 * 33 * sizeof(double));
    float* band = s_sh + align_up<float>(g.ns, 4);
    const int tid = threadIdx.x, bs = blockDim.x;
    const int BT = FA.band_tiles, BR = BT * TILE;
    const int tiles_y = g.ntiles / g.tiles_x;
    const int n_bands = (tiles_y + BT - 1) / BT;
    const int rows = BR + K - 1;  // band rows in the buffer
    if (blockIdx.x == 0 && tid == 0 && FA.status) FA.status[0] = cs.cstat[0];
    const bool bad = (cs.cstat[0] & ST_BADPARAM) != 0;
    int which = 0;
    for (int k = blockIdx.x; k < FA.n_src; k += gridDim.x) {
        __syncthreads();
        if (bad) {
            if (tid == 0) FA.chi2[k] = __longlong_as_double(0x7ff0000000000000LL);
            continue;
        }
        // stage the source (16-byte vectors when the row allows it)
        const float* src = FA.S + (long long)k * g.ns;
        if ((g.ns & 3) == 0 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            for (int i = tid; i < g.ns / 4; i += bs)
                reinterpret_cast<float4*>(s_sh)[i] = reinterpret_cast<const float4*>(src)[i];
        } else {
            for (int i = tid; i < g.ns; i += bs) s_sh[i] = src[i];
        }
        double chi = 0.0;
        for (int b = 0; b < n_bands; ++b) {
            __syncthreads();  // s staged / the previous band's convolution done
            // gather L s of padded rows [b BR, b BR + rows) into the band
            const int y0 = b * BR - g.hk;  // image row of band row 0
            for (int q = tid; q < rows * g.Wp; q += bs) {
                const int r = q / g.Wp, col = q - r * g.Wp;
                const int y = y0 + r, x = col - g.xoff;
                float val = 0.f;
                if (y >= 0 && y < g.ny && x >= 0 && x < g.nx) {
                    const int e = cs.inv[y * g.nx + x];
                    if (e >= 0) {
                        const Entry<float> en = cs.E[e];
                        const float* s0 = s_sh + en.base;
                        val = (1.f - en.v) * ((1.f - en.u) * s0[0] + en.u * s0[1]) +
                              en.v * ((1.f - en.u) * s0[g.sx] + en.u * s0[g.sx + 1]);
                    }
                }
                band[q] = val;
            }
            __syncthreads();
            // one 4x4 output tile per thread
            const int ty_l = tid / g.tiles_x, tx = tid - ty_l * g.tiles_x;
            const int ty = b * BT + ty_l;
            if (ty_l < BT && ty < tiles_y) {
                float o16[16];
                conv_tile_fast<K, TAPS_PARAM>(band + (ty_l * TILE) * g.Wp + tx * TILE, g.Wp, nullptr, FA.ptap, o16);
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const int y = ty * TILE + r;
                    const int pp = (y + g.hk) * g.Wp + tx * TILE + g.xoff;
                    const V4<float> sw = ld4(cs.swp + pp), dv = ld4(cs.dpad + pp);
#pragma unroll
                    for (int cc = 0; cc < TILE; ++cc) {
                        const double res = (double)sw.v[cc] * ((double)dv.v[cc] - (double)o16[r * 4 + cc]);
                        chi = fma(res, res, chi);
                        const int x = tx * TILE + cc;
                        if (FA.model && y < g.ny && x < g.nx)
                            FA.model[(long long)k * g.nx * g.ny + y * g.nx + x] = o16[r * 4 + cc];
                    }
                }
            }
        }
        const double cval = block_sum(chi, red, which);
        which ^= 1;
        if (tid == 0) FA.chi2[k] = cval;
    }
}

}  // namespace mirage
