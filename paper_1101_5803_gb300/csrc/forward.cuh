// Banded forward batch (FP32 contexts, one ray per pixel): model = B L s and
// Eq. chi2 for many sources at one lens (Section 3.2's refinement fitness).
//
// One CTA of FWD_THREADS threads per source at a time (persistent over the
// sources).  The source vector is staged in shared memory; the image is
// processed in bands of whole tile rows (two buffers: one band is filled
// while the previous one is convolved), each band's zero-padded L s values
// (its rows plus the K-1 halo rows) gathered straight into shared memory
// from a pixel-ordered map of the rays' cells and weights (k_pixmap), so
// L s never goes to global memory.  Each thread owns one 4x4 tile of the
// band and convolves it with the PSF taps (staged in shared memory, read as
// warp-uniform broadcasts), in a loop over pairs of tap rows (each input row is loaded once per pair; the
// loop body stays small enough for the instruction cache, which the fully
// unrolled 21x21 tile is not).  chi^2: FP32 per tile, FP64 across tiles.
#pragma once

#include "fast.cuh"

namespace mirage {

constexpr int FWD_THREADS = 512;
constexpr int MAX_FTAP = 31 * 31;

struct FwdArgs {
    const Prob<float>* probs;
    CandScratch<float> cs;
    const float4* pixmap;  // [npix] {cell base (int bits) or -1, u, v, 0} in pixel order
    const float* S;   // [n_src][ns]
    int n_src;
    float* model;     // nullable [n_src][npix]
    double* chi2;     // [n_src]
    int* status;      // nullable [1]
    int band_tiles;   // tile rows per band
};

// shared memory: taps, source vector, then two bands of (band rows + K - 1) x Wp
__host__ inline size_t fwd_band_smem(const Prob<float>& P, int band_tiles) {
    return 16 + 2 * 33 * sizeof(double) + align_up<float>(sizeof(float) * P.K * P.K, 16) +
           align_up<float>(sizeof(float) * P.ns, 16) +
           2 * sizeof(float) * (size_t)(band_tiles * TILE + P.K - 1) * P.Wp;
}

// pixel-ordered ray map of candidate 0 (one ray per pixel)
template <int UNUSED = 0>
__global__ void __launch_bounds__(NTHREADS) k_pixmap(const Prob<float>* __restrict__ probs, CandScratch<float> cs,
                                                   float4* __restrict__ pixmap) {
    const Prob<float>& P = probs[0];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.npix; j += gridDim.x * blockDim.x) {
        const int e = cs.inv[j];
        float4 m = make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
        if (e >= 0) {
            const Entry<float> en = cs.E[e];
            m = make_float4(__int_as_float(en.base), en.u, en.v, 0.f);
        }
        pixmap[j] = m;
    }
}

// One 4x4 output tile: out[r][c] = sum_{a,b} t[a][b] in[r + a][c + b + SHF]
// (t = the taps in shared memory), looping over pairs of tap rows: rows a..a+4 of
// the window serve tap rows a (output rows 0..3) and a+1 (output rows 0..3
// from window rows a+1..a+4).
template <int K>
__device__ __forceinline__ void conv_tile_pairs(const float* __restrict__ Pb, int Wp, const float* pt, float (&out)[16]) {
    constexpr int HK = (K - 1) / 2;
    constexpr int SHF = xoff_of<float>(HK) - HK;
    constexpr int W = TILE + K - 1 + SHF;
    constexpr int NVW = (W + 3) / 4 * 4;
    const unsigned src_a = smem_addr(Pb);
    float acc[TILE][TILE];
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int c = 0; c < TILE; ++c) acc[r][c] = 0.f;
#pragma unroll 1
    for (int a = 0; a + 1 < K; a += 2) {
#pragma unroll
        for (int rr = 0; rr <= TILE; ++rr) {
            float in[NVW];
#pragma unroll
            for (int v = 0; v < NVW; v += 4) lds_vec(src_a + (unsigned)(((a + rr) * Wp + v) * sizeof(float)), in + v);
#pragma unroll
            for (int b = 0; b < K; ++b) {
                if (rr < TILE) {
                    const float t = pt[a * K + b];
#pragma unroll
                    for (int c = 0; c < TILE; ++c) acc[rr][c] = fmaf(t, in[SHF + b + c], acc[rr][c]);
                }
                if (rr >= 1) {
                    const float t = pt[(a + 1) * K + b];
#pragma unroll
                    for (int c = 0; c < TILE; ++c) acc[rr - 1][c] = fmaf(t, in[SHF + b + c], acc[rr - 1][c]);
                }
            }
        }
    }
    if constexpr (K % 2 == 1) {  // the last tap row alone
        constexpr int a = K - 1;
#pragma unroll
        for (int rr = 0; rr < TILE; ++rr) {
            float in[NVW];
#pragma unroll
            for (int v = 0; v < NVW; v += 4) lds_vec(src_a + (unsigned)(((a + rr) * Wp + v) * sizeof(float)), in + v);
#pragma unroll
            for (int b = 0; b < K; ++b) {
                const float t = pt[a * K + b];
#pragma unroll
                for (int c = 0; c < TILE; ++c) acc[rr][c] = fmaf(t, in[SHF + b + c], acc[rr][c]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int c = 0; c < TILE; ++c) out[r * 4 + c] = acc[r][c];
}

template <int K>
__global__ void __launch_bounds__(FWD_THREADS, 1) k_forward_band(const __grid_constant__ FwdArgs FA) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob<float>& P = FA.probs[0];
    const CandScratch<float>& cs = FA.cs;
    const Geo<float> g = geo_of(P, cs.nent[0]);
    double* red = reinterpret_cast<double*>(smem + 16);
    float* taps = reinterpret_cast<float*>(smem + 16 + 2 * 33 * sizeof(double));
    float* s_sh = taps + align_up<float>(K * K, 4);
    float* band = s_sh + align_up<float>(g.ns, 4);
    const int tid = threadIdx.x, bs = blockDim.x;
    // taps of B: the flipped PSF, row-major K x K
    for (int i = tid; i < K * K; i += bs) {
        const int a = i / K, b = i - a * K;
        taps[i] = P.psf[(K - 1 - a) * K + (K - 1 - b)];
    }
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
        // band fill: L s of padded rows [b BR, b BR + rows) into dst, four
        // columns per step (row and column advanced without division)
        auto fill = [&](int b, float* dst) {
            const int y0 = b * BR - g.hk;  // image row of band row 0
            const int W4 = g.Wp >> 2, dr = bs / W4, dc = bs - dr * W4;
            int r = tid / W4, c4 = tid - (tid / W4) * W4;
            for (; r < rows;) {
                const int y = y0 + r;
                float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                if (y >= 0 && y < g.ny) {
                    float v4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int x = c4 * 4 + q - g.xoff;
                        v4[q] = 0.f;
                        if (x >= 0 && x < g.nx) {
                            const float4 m = FA.pixmap[y * g.nx + x];
                            const int base = __float_as_int(m.x);
                            if (base >= 0) {
                                const float* s0 = s_sh + base;
                                v4[q] = (1.f - m.z) * ((1.f - m.y) * s0[0] + m.y * s0[1]) +
                                        m.z * ((1.f - m.y) * s0[g.sx] + m.y * s0[g.sx + 1]);
                            }
                        }
                    }
                    val = make_float4(v4[0], v4[1], v4[2], v4[3]);
                }
                reinterpret_cast<float4*>(dst)[r * W4 + c4] = val;
                r += dr;
                c4 += dc;
                if (c4 >= W4) {
                    c4 -= W4;
                    ++r;
                }
            }
        };
        // two band buffers: while band b is convolved, band b + 1 is filled;
        // odd warps fill first, even warps convolve first, so the fill's
        // global loads wait while the other half of the warps keep the FMA
        // pipe busy
        const int bandsz = rows * g.Wp;
        const bool fill_first = ((tid >> 5) & 1) != 0;
        __syncthreads();  // s staged
        fill(0, band);
        double chi = 0.0;
        for (int b = 0; b < n_bands; ++b) {
            __syncthreads();  // band b filled; band b - 1's convolution done
            float* cur = band + (b & 1) * bandsz;
            float* nxt = band + ((b + 1) & 1) * bandsz;
            if (fill_first && b + 1 < n_bands) fill(b + 1, nxt);
            // one 4x4 output tile per thread; the chi^2 operands are loaded
            // before the convolution so that their latency overlaps it
            const int ty_l = tid / g.tiles_x, tx = tid - ty_l * g.tiles_x;
            const int ty = b * BT + ty_l;
            if (ty_l < BT && ty < tiles_y) {
                V4<float> sw[TILE], dv[TILE];
#pragma unroll
                for (int rr = 0; rr < TILE; ++rr) {
                    const int pp = (ty * TILE + rr + g.hk) * g.Wp + tx * TILE + g.xoff;
                    sw[rr] = ld4(cs.swp + pp);
                    dv[rr] = ld4(cs.dpad + pp);
                }
                float o16[16];
                conv_tile_pairs<K>(cur + (ty_l * TILE) * g.Wp + tx * TILE, g.Wp, taps, o16);
                float ct = 0.f;  // the tile's 16 terms in FP32, then one FP64 add
#pragma unroll
                for (int rr = 0; rr < TILE; ++rr) {
                    const int y = ty * TILE + rr;
#pragma unroll
                    for (int cc = 0; cc < TILE; ++cc) {
                        const float res = sw[rr].v[cc] * (dv[rr].v[cc] - o16[rr * 4 + cc]);
                        ct = fmaf(res, res, ct);
                        const int x = tx * TILE + cc;
                        if (FA.model && y < g.ny && x < g.nx)
                            FA.model[(long long)k * g.nx * g.ny + y * g.nx + x] = o16[rr * 4 + cc];
                    }
                }
                chi += (double)ct;
            }
            if (!fill_first && b + 1 < n_bands) fill(b + 1, nxt);
        }
        const double cval = block_sum(chi, red, which);
        which ^= 1;
        if (tid == 0) FA.chi2[k] = cval;
    }
}

}  // namespace mirage
