// Fast-path CGLS item kernel for small images (FP32 contexts).
//
// Same method as k_cgls (FP32 inner CGLS inside the FP64 residual
// refinement), laid out for two resident CTAs per SM:
//   * one ray per pixel and an identity or Laplacian H (square H);
//   * each thread owns exactly one 4x4 image tile (images up to 256 tiles)
//     and keeps that tile's residual, sqrt(W), q = sqrt(W) B L p and mapped
//     mask in registers; each thread also owns up to four source pixels
//     (i = tid + k * blockDim.x) and keeps their x, s and sqrt(lam) H p,
//     plus a bit mask of their occupied corner cells and existing neighbours;
//   * shared memory holds the two padded convolution buffers (P1 = L p,
//     reused for u = B^T sqrt(W) r at mapped pixels; P2 = sqrt(W) r, reused
//     for the four L^T corner planes), the rays in 12-byte form sorted by
//     cell, 16-bit cell starts, p and r_reg;
//   * L^T u is a balanced walk: every thread sums an equal run of the sorted
//     rays into per-cell corner totals; cells split between runs are joined
//     in a fixed order, so the result does not depend on scheduling;
//   * the convolution uses packed FP32x2 FMAs (__ffma2_rn) on tap pairs
//     stored duplicated in shared memory, or taps held as kernel parameters.
#pragma once

#include "kernels.cuh"

namespace mirage {

template <int K>
__device__ __forceinline__ void conv_tile_x2(const float* __restrict__ Pb, int Wp, const float2* __restrict__ taps2,
                                             float2 (&acc)[TILE][2]) {
    constexpr int HK = (K - 1) / 2;
    constexpr int SHF = xoff_of<float>(HK) - HK;
    constexpr int W = TILE + K - 1 + SHF;
    constexpr int NVW = (W + 3) / 4 * 4;
    const unsigned src_a = smem_addr(Pb);
    const unsigned tap_a = smem_addr(taps2);
#pragma unroll
    for (int r = 0; r < TILE; ++r) {
        acc[r][0] = make_float2(0.f, 0.f);
        acc[r][1] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < TILE + K - 1; ++i) {
        float in[NVW];
#pragma unroll
        for (int v = 0; v < NVW; v += 4) lds_vec(src_a + (unsigned)((i * Wp + v) * sizeof(float)), in + v);
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const int o = b + SHF;
            const float2 lo = make_float2(in[o], in[o + 1]);
            const float2 hi = make_float2(in[o + 2], in[o + 3]);
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int a = i - r;
                if (a >= 0 && a < K) {
                    float2 t;
                    asm("ld.shared.v2.f32 {%0, %1}, [%2];"
                        : "=f"(t.x), "=f"(t.y)
                        : "r"(tap_a + (unsigned)((a * K + b) * sizeof(float2))));
                    acc[r][0] = __ffma2_rn(t, lo, acc[r][0]);
                    acc[r][1] = __ffma2_rn(t, hi, acc[r][1]);
                }
            }
        }
    }
}

// Kernel arguments of the fast kernel: the common arguments plus, for
// launch groups that share one PSF, the taps themselves.  Kernel parameters
// live in the constant bank, which FFMA reads as a direct operand, so the
// unrolled convolution issues no tap loads at all.
constexpr int MAX_PTAP = 15 * 15;
struct FastArgs {
    CglsArgs<float> A;
    float ptap[2][MAX_PTAP];  // [0] flipped PSF (B), [1] PSF (B^T), row-major K x K
};

// tap source of the fast convolution; TAPS_PARAM_TF32 is TAPS_PARAM with
// both factors of every product rounded to TF32 (10-bit mantissa, the taps
// on the host, the image values here) and FP32 accumulation: the arithmetic
// of a TF32 tensor-core convolution, to measure its effect on the inner
// solves (the refinement's residual stays exact)
enum : int { TAPS_SMEM_X2 = 0, TAPS_PARAM = 1, TAPS_PARAM_X2 = 2, TAPS_PARAM_TF32 = 3 };

// round to TF32 (nearest, ties away from zero), returned as a float
__device__ __forceinline__ float tf32_round(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int K, int MODE>
__device__ __forceinline__ void conv_tile_fast(const float* __restrict__ Pb, int Wp, const float2* __restrict__ taps2,
                                               const float* __restrict__ pt, float (&out)[16]) {
    if constexpr (MODE == TAPS_SMEM_X2) {
        float2 acc[TILE][2];
        conv_tile_x2<K>(Pb, Wp, taps2, acc);
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            out[r * 4 + 0] = acc[r][0].x;
            out[r * 4 + 1] = acc[r][0].y;
            out[r * 4 + 2] = acc[r][1].x;
            out[r * 4 + 3] = acc[r][1].y;
        }
    } else {
        constexpr int HK = (K - 1) / 2;
        constexpr int SHF = xoff_of<float>(HK) - HK;
        constexpr int W = TILE + K - 1 + SHF;
        constexpr int NVW = (W + 3) / 4 * 4;
        const unsigned src_a = smem_addr(Pb);
        float2 acc2[TILE][2];
        float acc[TILE][TILE];
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            acc2[r][0] = acc2[r][1] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < TILE; ++c) acc[r][c] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < TILE + K - 1; ++i) {
            float in[NVW];
#pragma unroll
            for (int v = 0; v < NVW; v += 4) lds_vec(src_a + (unsigned)((i * Wp + v) * sizeof(float)), in + v);
            if constexpr (MODE == TAPS_PARAM_TF32) {
#pragma unroll
                for (int v = 0; v < NVW; ++v) in[v] = tf32_round(in[v]);
            }
#pragma unroll
            for (int b = 0; b < K; ++b) {
                const int o = b + SHF;
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const int a = i - r;
                    if (a >= 0 && a < K) {
                        const float t = pt[a * K + b];
                        if constexpr (MODE == TAPS_PARAM || MODE == TAPS_PARAM_TF32) {
#pragma unroll
                            for (int c = 0; c < TILE; ++c) acc[r][c] = fmaf(t, in[o + c], acc[r][c]);
                        } else {
                            const float2 t2 = make_float2(t, t);
                            acc2[r][0] = __ffma2_rn(t2, make_float2(in[o], in[o + 1]), acc2[r][0]);
                            acc2[r][1] = __ffma2_rn(t2, make_float2(in[o + 2], in[o + 3]), acc2[r][1]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            if constexpr (MODE == TAPS_PARAM || MODE == TAPS_PARAM_TF32) {
#pragma unroll
                for (int c = 0; c < TILE; ++c) out[r * 4 + c] = acc[r][c];
            } else {
                out[r * 4 + 0] = acc2[r][0].x;
                out[r * 4 + 1] = acc2[r][0].y;
                out[r * 4 + 2] = acc2[r][1].x;
                out[r * 4 + 3] = acc2[r][1].y;
            }
        }
    }
}

// Block sum of non-negative FP32 terms with one barrier, delivered to every
// thread of an NTHREADS block: a butterfly within each warp, then the warp
// sums along a fixed binary tree, so every thread holds the same value.
// Sums of non-negative terms have no cancellation, so plain FP32 additions
// keep ~log2(n) 2^-24 relative accuracy, far inside what the CG coefficients
// of an inner solve (which stops at a 1e-2 reduction) need.  `buf` holds
// 2 x 64 floats; alternate `half`.
__device__ __forceinline__ float block_sum_tree(float v, float* buf, int half) {
    constexpr int NW = NTHREADS / 32;
    float* b = buf + 64 * half;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) b[threadIdx.x >> 5] = v;
    __syncthreads();
    float x[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) x[i] = b[i];
#pragma unroll
    for (int st = 1; st < NW; st *= 2)
#pragma unroll
        for (int i = 0; i + st < NW; i += 2 * st) x[i] += x[i + st];
    return x[0];
}

// (H v)_i of the square regularisers (identity, or the five-point Laplacian
// with the neighbours that exist); nb = neighbour bits (1 left, 2 right,
// 4 below, 8 above).  The Laplacian is symmetric, so this is also H^T.
__device__ __forceinline__ float hrow_fast(const float* __restrict__ v, int i, unsigned nb, int sx, int reg) {
    if (reg != 2) return v[i];
    float a = 4.f * v[i];
    if (nb & 1u) a -= v[i - 1];
    if (nb & 2u) a -= v[i + 1];
    if (nb & 4u) a -= v[i - sx];
    if (nb & 8u) a -= v[i + sx];
    return a;
}

// Per-item constants of the fast kernel, written by thread 0 into shared
// memory (read back where needed instead of being held in registers).
struct FastItem {
    int nfz, top, mfr, W4;  // P2 frame float4s overlapped by the L^T planes
    int xl;                 // xoff / 4
    float inv_mfr;          // 1 / mfr
    float zero;             // 0: read in place of absent neighbours and cells
    // position in the current chain of lambdas (see ChainPos), kept here
    // rather than in registers; advanced by thread 0 between items
    int ch_c, ch_k, ch_last, ch_step, ch_warm, ch_prev_ok, ch_valid;
};
static_assert(sizeof(FastItem) <= 128, "fast-kernel item constants must fit the control slot");

constexpr int FAST_NPH = 12;  // per-phase clock slots (see mirage_last_phase_clocks)
constexpr size_t FAST_HDR = 16 + 2 * 33 * sizeof(double) + 128 + 16 * sizeof(unsigned long long);

// The refinement's FP64 convolution passes (conv64_pass's contract) on the
// FP32 pipe.  The taps are FP32 numbers, so the sums are double-float
// accumulations (dfloat.cuh): ~2^-44 relative instead of FP64's 2^-53, at
// about 11 FP32 operations per tap against one FP64 FMA (which the GPU
// issues at 1/64 of the FP32 rate).  hi and lo are staged in the
// two shared image buffers, which are cleared again afterwards (they must
// hold zeros outside the pixels each iteration writes).
template <int K>
__device__ __noinline__ double conv64_df(const double* __restrict__ src, float* __restrict__ hi,
                                         float* __restrict__ lo, const float2* __restrict__ taps,
                                         const float* __restrict__ swp, const float* __restrict__ dpad,
                                         float* __restrict__ rimg, double* __restrict__ Pb, double* __restrict__ Pc,
                                         const Geo<float> g, int mode) {
    for (int i = threadIdx.x; i < g.plen; i += blockDim.x) df_split(src[i], hi[i], lo[i]);
    __syncthreads();
    double ss = 0.0;
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
        const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
        const int base = (ty * TILE) * g.Wp + tx * TILE + g.sh;
#pragma unroll 1
        for (int r = 0; r < TILE; ++r) {
            float s[TILE], c[TILE];
#pragma unroll
            for (int q = 0; q < TILE; ++q) s[q] = c[q] = 0.f;
#pragma unroll 1
            for (int a = 0; a < K; ++a) {
                const float* hrow = hi + base + (r + a) * g.Wp;
                const float* lrow = lo + base + (r + a) * g.Wp;
                float xh[K + TILE - 1], xl[K + TILE - 1];
#pragma unroll
                for (int j = 0; j < K + TILE - 1; ++j) {
                    xh[j] = hrow[j];
                    xl[j] = lrow[j];
                }
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    const float tt = taps[a * K + b].x;
#pragma unroll
                    for (int q = 0; q < TILE; ++q) df_madd(s[q], c[q], tt, xh[b + q], xl[b + q]);
                }
            }
#pragma unroll
            for (int q = 0; q < TILE; ++q) {
                const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + q + g.xoff;
                const double v = (double)s[q] + (double)c[q];
                if (mode == 0) {
                    const double sw = (double)swp[pp];
                    const double res = sw * ((double)dpad[pp] - v);
                    rimg[pp] = (float)res;
                    Pb[pp] = sw * res;
                    ss += res * res;
                } else {
                    Pc[pp] = v;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < g.plen; i += blockDim.x) {
        hi[i] = 0.f;
        lo[i] = 0.f;
    }
    return ss;
}

// residual64's convolution functor for the two-CTA kernel
template <int K>
struct Conv64DF {
    float* hi;
    float* lo;
    const float2* taps;  // [0, K*K): flipped PSF (B); [K*K, 2 K*K): PSF (B^T)
    __device__ double operator()(const Work<float>& w, const Geo<float>& g, int mode) const {
        return conv64_df<K>(mode == 0 ? w.Pa : w.Pb, hi, lo, taps + (mode == 0 ? 0 : K * K), w.swp, w.dpad, w.rimg,
                            w.Pb, w.Pc, g, mode);
    }
};

template <int K, int NSP, int MODE>
__global__ void __launch_bounds__(NTHREADS, 2) k_cgls_fast(const __grid_constant__ FastArgs FA) {
    static_assert(NSP <= 4, "the per-thread masks describe at most four source pixels");
    using T = float;
    constexpr int bs = NTHREADS;
    const CglsArgs<float>& A = FA.A;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    double* red = reinterpret_cast<double*>(smem + 16);
    FastItem* fi = reinterpret_cast<FastItem*>(smem + 16 + 2 * 33 * sizeof(double));
    unsigned long long* phs = reinterpret_cast<unsigned long long*>(smem + 16 + 2 * 33 * sizeof(double) + 128);
    float* pbuf = reinterpret_cast<float*>(red);  // 2 x 64 floats for block_sum_tree
    int last_c = -1;
    int which = 0;
    // per-phase clocks (thread 0, kept in shared memory): 0 L p + H p,
    // 1 B conv, 2 delta reduction, 3 updates + residual store, 4 B^T conv,
    // 5 L^T ray walk, 6 L^T combination of split cells, 7 L^T gather + H^T,
    // 8 gamma reduction, 9 p update, 10 FP64 refinement, 11 item set-up
    const bool timed = A.phase_clk != nullptr && tid == 0;
    if (timed) {
        for (int i = 0; i < 15; ++i) phs[i] = 0ull;
        phs[15] = clock64();
    }
#define PHASE(n)                                   \
    do {                                           \
        if (timed) {                               \
            const unsigned long long t_ = clock64(); \
            phs[n] += t_ - phs[15];                \
            phs[15] = t_;                          \
        }                                          \
    } while (0)

    if (tid == 0) fi->ch_last = -1;
    while (true) {
        __syncthreads();
        if (tid == 0) {
            ChainPos ch;
            ch.c = fi->ch_c;
            ch.k = fi->ch_k;
            ch.k_last = fi->ch_last;
            ch.step = fi->ch_step;
            ch.prev_ok = fi->ch_prev_ok != 0;
            fi->ch_valid = 1;
            if (!ch.next()) {
                const int it_idx = atomicAdd(A.counter, 1);
                if (it_idx < A.n_items)
                    ch.start(A.items[it_idx]);
                else
                    fi->ch_valid = 0;
            }
            fi->ch_c = ch.c;
            fi->ch_k = ch.k;
            fi->ch_last = ch.k_last;
            fi->ch_step = ch.step;
            fi->ch_warm = ch.warm;
            fi->ch_prev_ok = ch.prev_ok;
        }
        __syncthreads();
        if (!fi->ch_valid) break;
        const int c = fi->ch_c, k = fi->ch_k;
        const Prob<T>& P = A.probs[A.cand_prob[c]];
        const CandScratch<T>& cs = A.cs;
        const int nent = cs.nent[c];
        const Geo<T> g = geo_of(P, nent);

        // ---- carve shared memory
        unsigned char* sp = smem + FAST_HDR;
        float2* taps2 = reinterpret_cast<float2*>(sp);
        sp += align_up<T>(sizeof(float2) * 2 * K * K, 16);
        Work<T> w;  // w.fft starts null (default member initialiser): the shared FP64 passes test it
        w.taps = nullptr;
        w.taps64 = reinterpret_cast<double*>(sp);
        sp += align_up<T>(sizeof(double) * 2 * K * g.kp, 16);
        float* P1 = reinterpret_cast<float*>(sp);
        sp += align_up<T>(sizeof(float) * g.plen, 16);
        float* P2 = reinterpret_cast<float*>(sp);
        sp += align_up<T>(sizeof(float) * g.plen, 16);
        unsigned* eidx = reinterpret_cast<unsigned*>(sp);
        sp += align_up<T>(sizeof(unsigned) * (size_t)P.nrays, 16);
        float2* euv = reinterpret_cast<float2*>(sp);
        sp += align_up<T>(sizeof(float2) * (size_t)P.nrays, 16);
        unsigned short* cst16 = reinterpret_cast<unsigned short*>(sp);
        sp += align_up<T>(sizeof(unsigned short) * (size_t)(P.ncells + 1), 16);
        float* p = reinterpret_cast<float*>(sp);
        sp += align_up<T>(sizeof(float) * g.ns, 16);
        float* rreg = reinterpret_cast<float*>(sp);
        sp += align_up<T>(sizeof(float) * g.nreg, 16);
        float* Sq = reinterpret_cast<float*>(sp);  // L^T partials of cells split across ranges: Sq[q * bs + t]
        sp += sizeof(float) * 4 * bs;

        // ---- global buffers: refinement (double) and its FP32 hand-over
        unsigned char* slab = reinterpret_cast<unsigned char*>(A.slab) + (long long)blockIdx.x * A.slab_stride;
        w.Pa = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.plen, 4);
        w.Pb = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.plen, 4);
        w.Pc = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.plen, 4);
        w.x64 = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.ns, 4);
        w.xb = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.ns, 4);
        w.h64 = reinterpret_cast<double*>(slab);
        slab += sizeof(double) * align_up<T>(g.nreg, 4);
        w.rimg = reinterpret_cast<float*>(slab);
        slab += sizeof(float) * align_up<T>(g.plen, 4);
        w.s = reinterpret_cast<float*>(slab);
        slab += sizeof(float) * align_up<T>(g.ns, 4);
        w.rreg = rreg;
        w.swp = const_cast<float*>(cs.swp + (long long)c * cs.sPad);
        w.dpad = cs.dpad + (long long)c * cs.sPad;
        w.E = nullptr;
        w.E64 = cs.E64 + (long long)c * cs.sE;
        w.inv = nullptr;
        w.cst = cs.cst + (long long)c * cs.sCst;

        if (c != last_c) {
            const Entry<T>* gE = cs.E + (long long)c * cs.sE;
            for (int i = tid; i < nent; i += bs) {
                const Entry<T> en = gE[i];
                eidx[i] = (unsigned)en.ppos | ((unsigned)en.base << 16);
                euv[i] = make_float2(en.u, en.v);
            }
            for (int i = tid; i <= P.ncells; i += bs) cst16[i] = (unsigned short)w.cst[i];
            for (int i = tid; i < 2 * K * K; i += bs) {
                const int h = i / (K * K), rem = i - h * K * K;
                const int a = rem / K, b = rem - a * K;
                const float v = h == 0 ? P.psf[(K - 1 - a) * K + (K - 1 - b)] : P.psf[a * K + b];
                taps2[i] = make_float2(v, v);
            }
            for (int i = tid; i < 2 * K * g.kp; i += bs) {
                const int h = i / (K * g.kp), rem = i - h * K * g.kp;
                const int a = rem / g.kp, b = rem - a * g.kp;
                double v = 0.0;
                if (b < K) v = h == 0 ? (double)P.psf[(K - 1 - a) * K + (K - 1 - b)] : (double)P.psf[a * K + b];
                w.taps64[i] = v;
            }
        }
        last_c = c;
        for (int i = tid; i < g.plen; i += bs) {
            P1[i] = 0.f;
            P2[i] = 0.f;
            w.Pa[i] = 0.0;
            w.Pb[i] = 0.0;
        }
        {
            if (tid == 0) {
                // the L^T planes occupy P2[0, 4 ns): its frame float4s there
                // (top frame rows, then the side margins of interior rows)
                // are cleared again before each B^T convolution
                const int W4 = g.Wp >> 2, tiles_y = g.ntiles / g.tiles_x;
                const int mfr = W4 - g.tiles_x;
                const int rows = max(0, min((4 * g.ns + g.Wp - 1) / g.Wp - g.hk, TILE * tiles_y));
                fi->W4 = W4;
                fi->mfr = mfr;
                fi->top = g.hk * W4;
                fi->nfz = g.hk * W4 + rows * mfr;
                fi->xl = g.xoff >> 2;
                fi->inv_mfr = mfr > 0 ? 1.f / (float)mfr : 0.f;
                fi->zero = 0.f;
            }
        }
        __syncthreads();

        // ---- tile ownership, sqrt(W) and mapped mask in registers
        const bool own = tid < g.ntiles;
        const int ty = own ? tid / g.tiles_x : 0, tx = own ? tid - (tid / g.tiles_x) * g.tiles_x : 0;
        const int pp0 = (ty * TILE + g.hk) * g.Wp + tx * TILE + g.xoff;
        // the tile holding this tile's pixels in the reversed image (L p is
        // stored reversed: pixel (Y, X) at (ny-1-Y, nx-1-X))
        const float* P1r = P1 + ((g.ntiles / g.tiles_x - 1 - ty) * TILE) * g.Wp + (g.tiles_x - 1 - tx) * TILE;
        const int crev = (P.ny - 1 + 2 * g.hk) * g.Wp + P.nx - 1 + 2 * g.xoff;  // ppos -> reversed ppos
        const float* P2t = P2 + (ty * TILE) * g.Wp + tx * TILE;
        float sw[16];
        unsigned mbits = 0;
        // L applied to ones marks the mapped pixels
        for (int e = tid; e < nent; e += bs) P1[eidx[e] & 0xffffu] = 1.f;
        __syncthreads();
        if (own) {
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const V4<float> m4 = ld4(P1 + pp0 + r * g.Wp);
                const V4<float> s4 = ld4(w.swp + pp0 + r * g.Wp);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    sw[r * 4 + cc] = s4.v[cc];
                    if (m4.v[cc] != 0.f) mbits |= 1u << (r * 4 + cc);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) sw[q] = 0.f;
        }
        __syncthreads();
        for (int i = tid; i < g.plen; i += bs) P1[i] = 0.f;

        // ---- per source pixel of this thread: which of its four corner
        // cells hold rays (bits 4kk..4kk+3: cells (ia, ib), (ia-1, ib),
        // (ia, ib-1), (ia-1, ib-1)) and which Laplacian neighbours exist
        // (bits 16+4kk..: left, right, below, above)
        unsigned msk = 0;
#pragma unroll
        for (int kk = 0; kk < NSP; ++kk) {
            const int i = tid + kk * bs;
            if (i < g.ns) {
                const int ib = i / g.sx, ia = i - ib * g.sx;
                const bool lf = ia >= 1, rt = ia <= g.sx - 2, dn = ib >= 1, up = ib <= g.sy - 2;
                const int cl = ib * g.ncx + ia;
                unsigned m = 0;
                if (rt && up && cst16[cl + 1] > cst16[cl]) m |= 1u;
                if (lf && up && cst16[cl] > cst16[cl - 1]) m |= 2u;
                if (rt && dn && cst16[cl - g.ncx + 1] > cst16[cl - g.ncx]) m |= 4u;
                if (lf && dn && cst16[cl - g.ncx] > cst16[cl - g.ncx - 1]) m |= 8u;
                const unsigned nb = (ia > 0 ? 1u : 0u) | (ia < g.sx - 1 ? 2u : 0u) | (ib > 0 ? 4u : 0u) |
                                    (ib < g.sy - 1 ? 8u : 0u);
                msk |= (m | (nb << 16)) << (4 * kk);
            }
        }
        // ---- this thread's ray range of the L^T walk.  Each warp takes a
        // span of the cell-sorted rays that starts and ends on a cell
        // boundary (nominally an eighth of them), cut into equal runs per
        // lane (of odd length, so that the lanes' reads fall on distinct
        // banks).  A cell split between runs therefore stays inside one warp
        // and its partials are joined by shuffles, with no block barrier.
        // wflags bit 0: this run's first cell continues from the previous run
        // (its partial is parked in Sq); bits 1..: how many later runs continue
        // this run's last cell (this lane adds their partials, in run order).
        int e0, e1, wflags = 0, jmax;
        {
            const int lane = tid & 31, wid = tid >> 5;
            // start of warp wq's span: the first cell boundary at or after its
            // nominal start
            auto span_start = [&](int wq) -> int {
                const int s0 = (int)(((long long)wq * nent) / (bs / 32));
                if (s0 <= 0 || s0 >= nent) return min(max(s0, 0), nent);
                const int b = (int)(eidx[s0] >> 16);  // lower-left source pixel of the ray's cell
                const int iy = b / g.sx;
                const int cell = iy * g.ncx + (b - iy * g.sx);
                return (int)cst16[cell] == s0 ? s0 : (int)cst16[cell + 1];
            };
            const int a0 = span_start(wid), a1 = span_start(wid + 1);
            const int Rw = ((a1 - a0 + 31) / 32) | 1;
            e0 = min(a0 + lane * Rw, a1);
            e1 = min(e0 + Rw, a1);
            int ncont = 0;
            if (e0 < e1) {
                const unsigned kf = eidx[e0] >> 16, kl = eidx[e1 - 1] >> 16;
                const bool cin = e0 > a0 && (eidx[e0 - 1] >> 16) == kf;
                if (!(cin && kf == kl))
                    for (int l2 = lane + 1; l2 < 32; ++l2) {
                        const int f2 = a0 + l2 * Rw;
                        if (f2 >= a1 || (eidx[f2] >> 16) != kl) break;
                        ++ncont;
                    }
                wflags = (cin ? 1 : 0) | (ncont << 1);
            }
            jmax = __reduce_max_sync(0xffffffffu, ncont);
        }
        __syncthreads();

        const int cstat = cs.cstat[c];
        const long long ok = (long long)c * A.max_lam + k;
        T* X = A.X + ok * A.max_ns;
        if (cstat & (ST_BADPARAM | ST_EMPTY)) {
            for (int i = tid; i < g.ns; i += bs) X[i] = 0;
            if (tid == 0) {
                A.chi2[ok] = (cstat & ST_BADPARAM) ? __longlong_as_double(0x7ff0000000000000LL) : 0.0;
                A.reg[ok] = 0.0;
                A.iters[ok] = 0;
                if (A.relres) A.relres[ok] = 0.0;
                if (A.istat) A.istat[ok] = cstat;
            }
            if (tid == 0) fi->ch_prev_ok = 0;
            continue;
        }

        const double lam = A.lambdas[(long long)c * A.max_lam + k];
        const float sl = (float)sqrt(lam);
        const int maxit = A.maxit > 0 ? A.maxit : 25 * g.ns;
        PHASE(11);

        // ---- ||rhs|| in FP64
        for (int t = tid; t < g.ntiles; t += bs) {
            const int ty2 = t / g.tiles_x, tx2 = t - ty2 * g.tiles_x;
            for (int r = 0; r < TILE; ++r) {
                const int pp = (ty2 * TILE + r + g.hk) * g.Wp + tx2 * TILE + g.xoff;
                for (int cc = 0; cc < TILE; ++cc) {
                    const double s = (double)w.swp[pp + cc];
                    w.Pb[pp + cc] = s * s * (double)w.dpad[pp + cc];
                }
            }
        }
        __syncthreads();
        const Conv64DF<K> conv_df{P1, P2, taps2};
        conv_df(w, g, 1);
        __syncthreads();
        double rs = 0;
        for (int i = tid; i < g.ns; i += bs) {
            const int ib = i / g.sx, ia = i - ib * g.sx;
            const double v = apply_LT_at<T, double, double, false>(g, w.E64, w.cst, w.Pc, ia, ib);
            rs += v * v;
        }
        const double rhsn = sqrt(block_sum(rs, red, which));
        which ^= 1;

        // ---- Jacobi preconditioner of the inner solves: an approximation of
        // diag(A~^T A~) = diag(L^T B^T W B L) + lam diag(H^T H), taking
        // diag(L^T B^T W B L)_i ~ sum_rays weight_i^2 omega(pixel), where
        // omega_p = diag(B^T W B)_p = sum_k psf_k^2 W_{p+k-c} (exact for a delta
        // PSF; the off-diagonal terms of B^T W B and the cross terms between
        // rays are dropped).  Any positive diagonal leaves the solution
        // unchanged; this one cuts the CGLS iterations two- to threefold.
        float minv[NSP];
        {
            // W of the owned tile into P1 (its frame is zero)
            if (own) {
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    V4<float> o;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) o.v[cc] = sw[r * 4 + cc] * sw[r * 4 + cc];
                    st4(P1 + pp0 + r * g.Wp, o);
                }
            }
            __syncthreads();
            float4* cellp = reinterpret_cast<float4*>(P2);
            const float2* ptap = taps2 + K * K;  // the PSF itself (B^T taps)
            for (int cell = tid; cell < g.ncells; cell += bs) {
                const int k0 = cst16[cell], k1 = cst16[cell + 1];
                float c00 = 0.f, c10 = 0.f, c01 = 0.f, c11 = 0.f;
                for (int e = k0; e < k1; ++e) {
                    const unsigned id = eidx[e];
                    const float2 uv = euv[e];
                    const float* wrow = P1 + (int)(id & 0xffffu) - g.hk * g.Wp - g.hk;
                    float om = 0.f;
#pragma unroll 1
                    for (int a = 0; a < K; ++a) {
#pragma unroll
                        for (int b = 0; b < K; ++b) {
                            const float f = ptap[a * K + b].x;
                            om = fmaf(f * f, wrow[a * g.Wp + b], om);
                        }
                    }
                    const float u1 = uv.x * uv.x, u0 = (1.f - uv.x) * (1.f - uv.x);
                    const float v1 = uv.y * uv.y, v0 = (1.f - uv.y) * (1.f - uv.y);
                    c00 = fmaf(u0 * v0, om, c00);
                    c10 = fmaf(u1 * v0, om, c10);
                    c01 = fmaf(u0 * v1, om, c01);
                    c11 = fmaf(u1 * v1, om, c11);
                }
                cellp[cell] = make_float4(c00, c10, c01, c11);
            }
            __syncthreads();
            const float* cp = reinterpret_cast<const float*>(cellp);
#pragma unroll
            for (int kk = 0; kk < NSP; ++kk) {
                const int i = tid + kk * bs;
                minv[kk] = 0.f;
                if (i < g.ns) {
                    const int ib = i / g.sx, ia = i - ib * g.sx;
                    float dsum = 0.f;
                    if (ib <= g.sy - 2 && ia <= g.sx - 2) dsum += cp[4 * (ib * g.ncx + ia) + 0];
                    if (ib <= g.sy - 2 && ia >= 1) dsum += cp[4 * (ib * g.ncx + ia - 1) + 1];
                    if (ib >= 1 && ia <= g.sx - 2) dsum += cp[4 * ((ib - 1) * g.ncx + ia) + 2];
                    if (ib >= 1 && ia >= 1) dsum += cp[4 * ((ib - 1) * g.ncx + ia - 1) + 3];
                    // diag(H^T H): 1 (identity) or 16 + number of neighbours (Laplacian)
                    float h = 1.f;
                    if (g.reg == 2)
                        h = 16.f + (float)((ia > 0) + (ia < g.sx - 1) + (ib > 0) + (ib < g.sy - 1));
                    minv[kk] = 1.f / (dsum + (float)lam * h);
                }
            }
            __syncthreads();
            for (int cell = tid; cell < g.ncells; cell += bs) cellp[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (own) {
#pragma unroll
                for (int r = 0; r < TILE; ++r) st4(P1 + pp0 + r * g.Wp, V4<float>{{0.f, 0.f, 0.f, 0.f}});
            }
            __syncthreads();
        }

        if (fi->ch_warm && fi->ch_prev_ok) {
            // w.x64 still holds the previous lambda's solution of this chain
        } else if (A.warm_x) {
            const T* x0 = A.warm_x + ok * A.max_ns;
            for (int i = tid; i < g.ns; i += bs) w.x64[i] = (double)x0[i];
        } else {
            for (int i = tid; i < g.ns; i += bs) w.x64[i] = 0.0;
        }
        __syncthreads();

        int status = 0, total_it = 0, slow = 0;
        double chi2 = 0, reg2 = 0, g64 = 0, rel64 = 0, prev_rel = 1e300;
        constexpr int MAX_OUTER = 16;
        const double eta_min = A.eta;
        const int nsv = g.ns, sxv = g.sx, regv = g.reg;
        float* Q = P2;  // L^T corner planes: Q[q * ns + base], q = 00, 10, 01, 11
        // signed offset of the shared zero from Q (both in the one shared
        // array): absent corner cells read it through an index select
        const int zq = (int)(&fi->zero - Q);
        bool reverted = false;
        for (int outer = 0;; ++outer) {
            PHASE(11);
            chi2 = residual64<T>(w, g, lam, red, which, reg2, g64, conv_df);
            PHASE(10);
            rel64 = rhsn > 0 ? sqrt(g64) / rhsn : 0.0;
            if (reverted) {  // the best iterate, evaluated again
                status |= ST_STAG;
                break;
            }
            if (outer > 0 && !(rel64 <= prev_rel)) {
                // the last correction raised the true residual: back to the
                // best iterate; the next pass evaluates it and stops
                for (int i = tid; i < g.ns; i += bs) w.x64[i] = w.xb[i];
                __syncthreads();
                reverted = true;
                continue;
            }
            if (!isfinite(rel64)) {
                status |= ST_BREAK;
                break;
            }
            if (!(rel64 > A.tol)) break;
            if (total_it >= maxit || outer >= MAX_OUTER) {
                status |= ST_MAXIT;
                break;
            }
            slow = (outer > 0 && rel64 > 0.9 * prev_rel) ? slow + 1 : 0;
            if (slow >= 2) {
                status |= ST_STAG;
                break;
            }
            prev_rel = rel64;  // accepted residuals decrease: this is the best iterate
            for (int i = tid; i < g.ns; i += bs) w.xb[i] = w.x64[i];
            const double target = fmax(eta_min, fmin(MAX_TARGET, FINAL_MARGIN * A.tol / rel64));

            // ---- inner solve of the correction equation A d = r: Jacobi-
            // preconditioned CG on the normal equations (r = the FP64 residual
            // rounded to FP32, A = L^T B^T W B L + lam H^T H applied in FP32),
            // started from d = 0.  Every vector of the recursion is of the size
            // of the correction itself, so FP32 rounding stays relative to it
            // (an image-space CGLS residual would carry the data misfit, which
            // is ~1e7 times larger near convergence, into every gradient).
            float x[NSP], gv[NSP], z[NSP], hth[NSP];
            float gs = 0.f;
            const float lamf = (float)lam;
#pragma unroll
            for (int kk = 0; kk < NSP; ++kk) {
                const int i = tid + kk * bs;
                x[kk] = 0.f;
                gv[kk] = 0.f;
                z[kk] = 0.f;
                if (i < nsv) {
                    gv[kk] = w.s[i];
                    z[kk] = minv[kk] * gv[kk];
                    p[i] = z[kk];
                    gs = fmaf(gv[kk], z[kk], gs);
                }
            }
            float* hbuf = rreg;  // H p of the current direction (the CGLS residual slot is free here)
            int half = 0, it_in = 0, best_it = 0, brk = 0, stop = 0;
            float gam, g0, best = 1.f;
            {
                gam = block_sum_tree(gs, pbuf, half);  // its barrier also completes p
                half ^= 1;
                g0 = gam;
                brk = !isfinite(gam);
                stop = brk || !(gam > 0.f) || total_it >= maxit;
            }
            const int stag_window = max(4000, 2 * nsv);
            while (!stop) {
                // P1 <- L p at the mapped pixels, reversed, four rays at a time (all
                // loads first, so their latencies overlap); q_reg = sqrt(lam) H p
                for (int e = tid; e < nent; e += 4 * bs) {
                    unsigned id[4];
                    float2 uv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int ej = e + j * bs < nent ? e + j * bs : e;
                        id[j] = eidx[ej];
                        uv[j] = euv[ej];
                    }
                    float val[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float* s0 = p + (id[j] >> 16);
                        val[j] = (1.f - uv[j].y) * ((1.f - uv[j].x) * s0[0] + uv[j].x * s0[1]) +
                                 uv[j].y * ((1.f - uv[j].x) * s0[sxv] + uv[j].x * s0[sxv + 1]);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (e + j * bs < nent) P1[crev - (int)(id[j] & 0xffffu)] = val[j];
                }
                // H p of the owned source pixels into hbuf, and lam ||H p||^2
                float dh = 0.f;
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    if (i < nsv) {
                        const float h = hrow_fast(p, i, msk >> (16 + 4 * kk), sxv, regv);
                        hbuf[i] = h;
                        dh = fmaf(h, h, dh);
                    }
                }
                __syncthreads();
                PHASE(0);
                // q = B P1 on the owned tile: delta += ||sqrt(W) q||^2, P2 <- W q
                // B and B^T run one copy of the convolution code (one unrolled
                // K x K tile loop in the instruction cache instead of two).  L p
                // is stored reversed; B L p at a pixel is the PSF correlation of
                // the reversed image at the reversed pixel, so it is read from
                // the reversed tile in reversed order.  B^T is the PSF
                // correlation itself
                float dl_part = lamf * dh;
                float a = 0.f;
#pragma unroll 1
                for (int dir = 0; dir < 2; ++dir) {
                    float o16[16];
                    if (own) conv_tile_fast<K, MODE>(dir == 0 ? P1r : P2t, g.Wp, taps2 + K * K, FA.ptap[1], o16);
                    if (dir == 0) {
                        // q = sqrt(W) B L p on the owned tile: delta += ||q||^2, P2 <- W B L p
                        if (own) {
#pragma unroll
                            for (int r = 0; r < TILE; ++r) {
                                V4<float> o;
#pragma unroll
                                for (int cc = 0; cc < 4; ++cc) {
                                    const float t = sw[r * 4 + cc] * o16[(TILE - 1 - r) * 4 + (3 - cc)];
                                    dl_part = fmaf(t, t, dl_part);
                                    o.v[cc] = sw[r * 4 + cc] * t;
                                }
                                st4(P2 + pp0 + r * g.Wp, o);
                            }
                        }
                    // the previous L^T planes overwrote part of P2's zero frame
                    {
                        const int nfz = fi->nfz, top = fi->top;
                        for (int f = tid; f < nfz; f += bs) {
                            int q4 = f;
                            if (f >= top) {
                                const int f2 = f - top, mfr = fi->mfr, xl = fi->xl;
                                const int r = (int)(((float)f2 + 0.5f) * fi->inv_mfr);
                                const int j = f2 - r * mfr;
                                q4 = (g.hk + r) * fi->W4 + (j < xl ? j : j + g.tiles_x);
                            }
                            reinterpret_cast<float4*>(P2)[q4] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                    // H^T (H p) of the owned source pixels (neighbours' H p from hbuf)
    #pragma unroll
                    for (int kk = 0; kk < NSP; ++kk) {
                        const int i = tid + kk * bs;
                        hth[kk] = i < nsv ? hrow_fast(hbuf, i, msk >> (16 + 4 * kk), sxv, regv) : 0.f;
                    }
                        PHASE(1);
                        // delta = p^T A p; the reduction's barrier also completes P2
                        const float delta = block_sum_tree(dl_part, pbuf, half);
                        half ^= 1;
                        PHASE(2);
                        if (!(delta > 0.f) || !isfinite(delta)) {
                            brk = 1;
                            break;
                        }
                        a = gam / delta;
                    } else {
                        // u = B^T P2 on the owned tile, stored into P1 at mapped pixels
                        if (own) {
#pragma unroll
                            for (int r = 0; r < TILE; ++r) {
                                float* dst = P1 + pp0 + r * g.Wp;
#pragma unroll
                                for (int cc = 0; cc < 4; ++cc)
                                    if (mbits & (1u << (r * 4 + cc))) dst[cc] = o16[r * 4 + cc];
                            }
                        }
                        __syncthreads();  // u complete
                        PHASE(4);
                    }
                }
                if (brk) break;
                // L^T u: each lane walks its run of consecutive rays (sorted by
                // cell) and sums, per cell, the four corner weights times u; a
                // cell's total goes to the planes (indexed by the cell's base
                // source pixel), the partial of a cell continued from the
                // previous run to Sq.  The next ray is loaded before the current
                // one is used, and the sums are stored at the last ray of each
                // cell run (known from the next ray's cell)
                if (e0 < e1) {
                    // the ray index is loaded two rays ahead, so that the next
                    // ray's u load does not wait on an index loaded in the same
                    // iteration
                    unsigned id = eidx[e0];
                    unsigned idn = eidx[min(e0 + 1, e1 - 1)];
                    unsigned cur = id >> 16;
                    float* dst = (wflags & 1) ? Sq + tid : Q + cur;
                    int ps = (wflags & 1) ? bs : nsv;
                    float2 uv = euv[e0];
                    float U = P1[id & 0xffffu];
                    float c00 = 0.f, c10 = 0.f, c01 = 0.f, c11 = 0.f;
                    for (int e = e0; e < e1; ++e) {
                        const int en = min(e + 1, e1 - 1);
                        const unsigned idnn = eidx[min(e + 2, e1 - 1)];
                        const float2 uvn = euv[en];
                        const float Un = P1[idn & 0xffffu];
                        const unsigned key = id >> 16;
                        if (key != cur) {  // a new cell: its sums go to the planes
                            cur = key;
                            dst = Q + key;
                            ps = nsv;
                            c00 = c10 = c01 = c11 = 0.f;
                        }
                        const float uU = uv.x * U, u0 = U - uU;  // u U, (1-u) U
                        c00 = fmaf(1.f - uv.y, u0, c00);
                        c10 = fmaf(1.f - uv.y, uU, c10);
                        c01 = fmaf(uv.y, u0, c01);
                        c11 = fmaf(uv.y, uU, c11);
                        if (e == e1 - 1 || (idn >> 16) != key) {
                            dst[0] = c00;
                            dst[ps] = c10;
                            dst[2 * ps] = c01;
                            dst[3 * ps] = c11;
                        }
                        id = idn;
                        idn = idnn;
                        uv = uvn;
                        U = Un;
                    }
                }
                // join of split cells inside the warp: each run's parked
                // first-cell partial (this lane's own Sq slot, so no barrier)
                // is shuffled down to the lane owning that cell, which adds the
                // partials in run order (a fixed order: deterministic)
                if (jmax > 0) {
                    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
                    if (wflags & 1) {
                        f0 = Sq[tid];
                        f1 = Sq[bs + tid];
                        f2 = Sq[2 * bs + tid];
                        f3 = Sq[3 * bs + tid];
                    }
                    const int nc = wflags >> 1;
                    unsigned kl = 0;
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                    if (nc) {
                        kl = eidx[e1 - 1] >> 16;
                        a0 = Q[kl];
                        a1 = Q[nsv + kl];
                        a2 = Q[2 * nsv + kl];
                        a3 = Q[3 * nsv + kl];
                    }
                    for (int j = 1; j <= jmax; ++j) {
                        const float v0 = __shfl_down_sync(0xffffffffu, f0, j);
                        const float v1 = __shfl_down_sync(0xffffffffu, f1, j);
                        const float v2 = __shfl_down_sync(0xffffffffu, f2, j);
                        const float v3 = __shfl_down_sync(0xffffffffu, f3, j);
                        if (j <= nc) {
                            a0 += v0;
                            a1 += v1;
                            a2 += v2;
                            a3 += v3;
                        }
                    }
                    if (nc) {
                        Q[kl] = a0;
                        Q[nsv + kl] = a1;
                        Q[2 * nsv + kl] = a2;
                        Q[3 * nsv + kl] = a3;
                    }
                }
                __syncthreads();
                PHASE(5);
                // u has been read: clear the owned tile of P1 (the reversed L p
                // of the next iteration writes only mapped pixels)
                if (own) {
#pragma unroll
                    for (int r = 0; r < TILE; ++r) st4(P1 + pp0 + r * g.Wp, V4<float>{{0.f, 0.f, 0.f, 0.f}});
                }
                // pass 3: per source pixel, (A p)_i = the fixed-order sum of the
                // corners it receives from its (up to) four occupied cells plus
                // lam (H^T H p)_i; then the CG updates of x, g and z = M^-1 g
                float gsum = 0.f;
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    if (i < nsv) {
                        const unsigned m = msk >> (4 * kk);
                        // empty or absent cells read the shared zero: no branches,
                        // four independent loads; adding +0 changes nothing
                        const int q0 = (m & 1u) ? i : zq;
                        const int q1 = (m & 2u) ? nsv + i - 1 : zq;
                        const int q2 = (m & 4u) ? 2 * nsv + i - sxv : zq;
                        const int q3 = (m & 8u) ? 3 * nsv + i - sxv - 1 : zq;
                        float acc = 0.f;
                        acc += Q[q0];
                        acc += Q[q1];
                        acc += Q[q2];
                        acc += Q[q3];
                        const float ap = fmaf(lamf, hth[kk], acc);
                        x[kk] = fmaf(a, p[i], x[kk]);
                        gv[kk] = fmaf(-a, ap, gv[kk]);
                        z[kk] = minv[kk] * gv[kk];
                        gsum = fmaf(gv[kk], z[kk], gsum);
                    }
                }
                PHASE(7);
                const float gnew = block_sum_tree(gsum, pbuf, half);
                half ^= 1;
                PHASE(8);
                const float bt = gnew / gam;
                gam = gnew;
                ++it_in;
                ++total_it;
                {
                    // every thread takes the same decision from the same values
                    const float rel = sqrtf(gnew / g0);
                    if (!isfinite(gnew)) {
                        brk = 1;
                        stop = 1;
                    } else if (!(rel > (float)target) || total_it >= maxit) {
                        stop = 1;
                    } else if (rel < 0.5f * best) {
                        best = rel;
                        best_it = it_in;
                    } else if (it_in - best_it > stag_window) {
                        stop = 1;
                    }
                }
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    if (i < nsv) p[i] = fmaf(bt, p[i], z[kk]);
                }
                __syncthreads();
                PHASE(9);
            }
            if (brk) {
                status |= ST_BREAK;
                break;
            }
#pragma unroll
            for (int kk = 0; kk < NSP; ++kk) {
                const int i = tid + kk * bs;
                if (i < nsv) w.x64[i] += (double)x[kk];
            }
            // the inner loop leaves u in P1 at mapped pixels (L p overwrites
            // every one of them) and the L^T planes in P2 (the frame is
            // cleared again after the next B convolution)
            __syncthreads();
        }

        for (int i = tid; i < g.ns; i += bs) X[i] = (T)w.x64[i];
        if (tid == 0) {
            A.chi2[ok] = chi2;
            A.reg[ok] = reg2;
            A.iters[ok] = total_it;
            if (A.relres) A.relres[ok] = rel64;
            if (A.istat) A.istat[ok] = status | cstat;
        }
        if (tid == 0) fi->ch_prev_ok = !(status & ST_BREAK);
    }
    if (timed)
        for (int i = 0; i < FAST_NPH; ++i) atomicAdd(A.phase_clk + i, phs[i]);
#undef PHASE
}

// shared memory of the fast variant (0 if the problem is not eligible):
// one ray per pixel, a square regulariser, at most four source pixels and
// one image tile per thread, 16-bit ray/pixel/cell indices, and room for the
// four L^T corner planes (4 ns floats) in P2 above its last interior row
__host__ inline size_t fast_smem_bytes(const Prob<float>& P) {
    // (image sides in whole tiles: L p is stored reversed, and the reversed
    // image must fall on the same tile grid)
    if (P.Np != 1 || P.ntiles > NTHREADS || P.plen >= 65536 || P.nrays >= 65536 || P.ns > 4 * NTHREADS ||
        P.nreg != P.ns || 4 * P.ncells > P.plen || 4 * P.ns > (P.hk + TILE * P.tiles_y) * P.Wp ||
        P.nx % TILE != 0 || P.ny % TILE != 0)
        return 0;
    size_t o = FAST_HDR;
    o += align_up<float>(sizeof(float2) * 2 * P.K * P.K, 16);
    o += align_up<float>(sizeof(double) * 2 * P.K * P.kp, 16);
    o += 2 * align_up<float>(sizeof(float) * P.plen, 16);
    o += align_up<float>(sizeof(unsigned) * (size_t)P.nrays, 16);
    o += align_up<float>(sizeof(float2) * (size_t)P.nrays, 16);
    o += align_up<float>(sizeof(unsigned short) * (size_t)(P.ncells + 1), 16);
    o += align_up<float>(sizeof(float) * P.ns, 16);
    o += align_up<float>(sizeof(float) * P.nreg, 16);
    o += sizeof(float) * 4 * NTHREADS;
    return o;
}

__host__ inline size_t fast_slab_bytes(const Prob<float>& P) {
    size_t o = sizeof(double) * (3 * align_up<float>(P.plen, 4) + 2 * align_up<float>(P.ns, 4) + align_up<float>(P.nreg, 4));
    o += sizeof(float) * (align_up<float>(P.plen, 4) + align_up<float>(P.ns, 4));
    return align_up<float>(o, 256);
}

}  // namespace mirage
