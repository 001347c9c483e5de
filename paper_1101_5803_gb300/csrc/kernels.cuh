// Device code of the lens-inversion inner loop (sm_103a).
//
//   k_raytrace   Eq. thinlens + Eqs. SIEX/SIEY (+ external shear): every
//                (sub-)pixel ray is traced once per candidate; its bilinear
//                cell and weights (Section 2.2) are stored sorted by source
//                cell (stable in ray order), which gives a deterministic
//                gather form of L^T.  Also writes sqrt(W) = m / sigma and
//                sqrt(W) d in the padded image layout.
//   k_cgls       CGLS (Sections 2.2, 2.4) on min ||sqrt(W)(B L s - d)||^2 +
//                lambda ||H s||^2, i.e. CG on the normal equations of
//                Eq. TKReg, one (candidate, lambda) work item per CTA pass,
//                items pulled from a queue by a persistent grid.  L, B, B^T,
//                L^T and H are applied matrix-free; B and B^T are direct
//                zero-padded convolutions on 4x4 register tiles.
//   k_finalize   L-curve corner (Section 2.6) per candidate, status, s_out.
//   k_forward    B L s and Eq. chi2 for a batch of sources at one lens.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mirage {

constexpr int TILE = 4;        // each thread owns TILE x TILE image pixels in the convolutions
constexpr int NTHREADS = 256;  // CTA size of the item kernels
constexpr int MAX_LAM = 64;    // longest lambda grid of one candidate

enum : int { ST_MAXIT = 1, ST_STAG = 2, ST_BREAK = 4, ST_BADPARAM = 8, ST_EMPTY = 16, ST_FLAT = 32 };

// One mapped (sub-)pixel ray, stored sorted by source cell.
//   ppos : padded-layout position of its image pixel
//   base : source index of the lower-left centre of its cell
//   u, v : fractional position in the cell
template <typename T>
struct alignas(2 * sizeof(T) > 8 ? 2 * sizeof(T) : 16) Entry {
    int ppos;
    int base;
    T u;
    T v;
};

// Per-problem constants (device copy).
template <typename T>
struct Prob {
    int nx, ny, npix, sx, sy, ns, nreg, K, hk, n_sub, Np, nrays, ncx, ncells, reg;
    int Wp, Hp, plen, tiles_x, tiles_y, ntiles, kp;  // padded layout, tap row pitch
    T pix, cx, cy, sub0, subd, c0x, c0y, inv_hx, inv_hy, invNp;
    const T* d;
    const T* sigma;
    const uint8_t* mask;
    const T* psf;
};

// Per-candidate scratch written by k_raytrace (strides in elements).
template <typename T>
struct CandScratch {
    Entry<T>* E;      // [n_cand][sE]  sorted mapped rays
    Entry<T>* Etmp;   // [n_cand][sE]  rays in ray order (build only)
    int* inv;         // [n_cand][sInv] ray -> sorted position, -1 unmapped
    int* cst;         // [n_cand][sCst] cell start offsets (ncells + 1)
    T* swp;           // [n_cand][sPad] m / sigma in padded layout
    T* bwp;           // [n_cand][sPad] m d / sigma in padded layout
    int* nent;        // [n_cand]
    int* cstat;       // [n_cand]
    long long sE, sInv, sCst, sPad;
};

template <typename T>
struct CglsArgs {
    const Prob<T>* probs;
    const int* cand_prob;   // [n_cand]
    const double* lens;     // [n_cand][7]
    const double* lambdas;  // [n_cand][max_lam]
    const int* items;       // [n_items] packed c * MAX_LAM + k
    int n_items;
    int* counter;           // queue head
    double tol;
    int maxit;              // <= 0: 10 * ns
    int replace_every;
    int max_lam, max_ns;
    const T* warm_x;        // nullable [n_cand][max_lam][max_ns]
    CandScratch<T> cs;
    T* slab;                // BIG variant: per-CTA global work buffers
    long long slab_stride;
    T* X;                   // [n_cand][max_lam][max_ns]
    double* chi2;           // [n_cand][max_lam]
    double* reg;
    int* iters;
    double* relres;
    int* istat;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ float m_atanh(float x) { return atanhf(x); }
__device__ __forceinline__ double m_atanh(double x) { return atanh(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};

__device__ __forceinline__ void vload(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void vload(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
}

// explicit shared-memory loads (the tile code runs in a non-inlined
// function, where the compiler cannot infer the address space itself)
__device__ __forceinline__ void lds_vec(unsigned a, float* o) {
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(a));
}
__device__ __forceinline__ void lds_vec(unsigned a, double* o) {
    asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "r"(a));
}
__device__ __forceinline__ float lds_one(unsigned a, float) {
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_one(unsigned a, double) {
    double v;
    asm("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum.  `red` holds 2 x 33 doubles; callers alternate the
// halves (`which`) so consecutive reductions need one barrier pair each.
__device__ __forceinline__ double block_sum(double v, double* red, int which) {
    double* r = red + 33 * which;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) r[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = (lane < (int)(blockDim.x >> 5)) ? r[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) r[32] = t;
    }
    __syncthreads();
    return r[32];
}

// ---------------------------------------------------------------------------
// lens model
// ---------------------------------------------------------------------------
template <typename T>
struct LensT {
    T b, q, c, s, x0, y0, g1, g2, bqf, f;
    int sis, bad;
};

template <typename T>
__device__ LensT<T> make_lens(const double* l) {
    const double b = l[0], q = l[1], phi = l[2], x0 = l[3], y0 = l[4], g = l[5], tg = l[6];
    LensT<T> L;
    const bool fin = isfinite(b) && isfinite(q) && isfinite(phi) && isfinite(x0) && isfinite(y0) &&
                     isfinite(g) && isfinite(tg);
    L.bad = !(fin && b >= 0.0 && q > 0.0 && q <= 1.0);
    double cp = 1.0, sp = 0.0, c2 = 1.0, s2 = 0.0;
    if (!L.bad) {
        sincos(phi, &sp, &cp);
        sincos(2.0 * tg, &s2, &c2);
    }
    L.b = (T)b;
    L.q = (T)q;
    L.c = (T)cp;
    L.s = (T)sp;
    L.x0 = (T)x0;
    L.y0 = (T)y0;
    L.g1 = (T)(g * c2);
    L.g2 = (T)(g * s2);
    L.sis = (q >= 1.0 - 1e-6) ? 1 : 0;
    const double f = L.bad ? 0.0 : sqrt(fmax(0.0, 1.0 - q * q));
    L.f = (T)f;
    L.bqf = (T)((L.sis || L.bad) ? 0.0 : b * q / f);
    return L;
}

// Eq. thinlens with the SIE of Eqs. SIEX/SIEY (s = 0) rotated by phi about
// (x0, y0) plus external shear about the same centre.
template <typename T>
__device__ __forceinline__ void trace_ray(const LensT<T>& L, T tx, T ty, T& bx, T& by) {
    const T dx = tx - L.x0, dy = ty - L.y0;
    const T xl = L.c * dx + L.s * dy;
    const T yl = -L.s * dx + L.c * dy;
    T axl = 0, ayl = 0;
    if (L.sis) {
        const T r = m_sqrt(xl * xl + yl * yl);
        if (r > 0) {
            axl = L.b * xl / r;
            ayl = L.b * yl / r;
        }
    } else {
        const T psi = m_sqrt(L.q * L.q * xl * xl + yl * yl);
        if (psi > 0) {
            axl = L.bqf * m_atan(xl * L.f / psi);
            ayl = L.bqf * m_atanh(yl * L.f / psi);
        }
    }
    const T ax = L.c * axl - L.s * ayl + L.g1 * dx + L.g2 * dy;
    const T ay = L.s * axl + L.c * ayl + L.g2 * dx - L.g1 * dy;
    bx = tx - ax;
    by = ty - ay;
}

// ---------------------------------------------------------------------------
// k_raytrace: one CTA per candidate
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_raytrace(const Prob<T>* __restrict__ probs,
                                                       const int* __restrict__ cand_prob,
                                                       const double* __restrict__ lens, int cand0,
                                                       int n_cand, CandScratch<T> cs) {
    const int c = cand0 + blockIdx.x;
    if (c >= cand0 + n_cand) return;
    const Prob<T>& P = probs[cand_prob[c]];
    extern __shared__ int sh_counts[];  // [ncells] counts, then starts/cursors
    __shared__ int s_active, s_chunk[NTHREADS];

    Entry<T>* E = cs.E + (long long)c * cs.sE;
    Entry<T>* Et = cs.Etmp + (long long)c * cs.sE;
    int* inv = cs.inv + (long long)c * cs.sInv;
    int* cst = cs.cst + (long long)c * cs.sCst;
    T* swp = cs.swp + (long long)c * cs.sPad;
    T* bwp = cs.bwp + (long long)c * cs.sPad;
    const int tid = threadIdx.x, bs = blockDim.x;
    const LensT<T> L = make_lens<T>(lens + 7LL * c);

    for (int i = tid; i < P.plen; i += bs) {
        swp[i] = 0;
        bwp[i] = 0;
    }
    for (int i = tid; i < P.ncells; i += bs) sh_counts[i] = 0;
    if (tid == 0) s_active = 0;
    __syncthreads();

    if (L.bad) {
        for (int r = tid; r < P.nrays; r += bs) inv[r] = -1;
        for (int i = tid; i <= P.ncells; i += bs) cst[i] = 0;
        if (tid == 0) {
            cs.nent[c] = 0;
            cs.cstat[c] = ST_BADPARAM;
        }
        return;
    }

    // pass 1: trace every ray once, count rays per cell, build sqrt(W)
    const T half_x = (T)0.5 * (T)(P.nx - 1), half_y = (T)0.5 * (T)(P.ny - 1);
    const T fxmax = (T)(P.sx - 1), fymax = (T)(P.sy - 1);
    int my_active = 0;
    for (int j = tid; j < P.npix; j += bs) {
        const int x = j % P.nx, y = j / P.nx;
        const T tx = P.cx + ((T)x - half_x) * P.pix;
        const T ty = P.cy + ((T)y - half_y) * P.pix;
        const int pp = (y + P.hk) * P.Wp + x + P.hk;
        bool any = false;
        for (int a = 0; a < P.Np; ++a) {
            const int ax = a % P.n_sub, ay = a / P.n_sub;
            T bx, by;
            trace_ray(L, tx + P.sub0 + (T)ax * P.subd, ty + P.sub0 + (T)ay * P.subd, bx, by);
            const T fx = (bx - P.c0x) * P.inv_hx;
            const T fy = (by - P.c0y) * P.inv_hy;
            const bool m = (fx >= (T)0) && (fx <= fxmax) && (fy >= (T)0) && (fy <= fymax);
            Entry<T> e;
            e.ppos = pp;
            if (m) {
                const int ix0 = min((int)m_floor(fx), P.sx - 2);
                const int iy0 = min((int)m_floor(fy), P.sy - 2);
                e.base = iy0 * P.sx + ix0;
                e.u = fx - (T)ix0;
                e.v = fy - (T)iy0;
                atomicAdd(&sh_counts[iy0 * P.ncx + ix0], 1);
                any = true;
            } else {
                e.base = -1;
                e.u = 0;
                e.v = 0;
            }
            Et[(long long)j * P.Np + a] = e;
        }
        const T w = (any && P.mask[j]) ? (T)1 / P.sigma[j] : (T)0;
        swp[pp] = w;
        bwp[pp] = w * P.d[j];
        my_active += (w != (T)0);
    }
    if (my_active) atomicAdd(&s_active, my_active);
    __syncthreads();

    // exclusive scan of the cell counts (chunk per thread, then the chunk sums)
    const int chunk = (P.ncells + bs - 1) / bs;
    const int lo = min(tid * chunk, P.ncells), hi = min(lo + chunk, P.ncells);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += sh_counts[i];
    s_chunk[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int t = 0; t < bs; ++t) {
            const int v = s_chunk[t];
            s_chunk[t] = run;
            run += v;
        }
        cst[P.ncells] = run;
        cs.nent[c] = run;
        cs.cstat[c] = (s_active > 0) ? 0 : ST_EMPTY;
    }
    __syncthreads();
    int run = s_chunk[tid];
    for (int i = lo; i < hi; ++i) {
        const int v = sh_counts[i];
        sh_counts[i] = run;
        cst[i] = run;
        run += v;
    }
    __syncthreads();

    // pass 2: one warp places the rays in ray order (stable within a cell)
    if (tid < 32) {
        const int lane = tid;
        const unsigned lt = (1u << lane) - 1u;
        for (int r0 = 0; r0 < P.nrays; r0 += 32) {
            const int r = r0 + lane;
            Entry<T> e;
            e.base = -1;
            if (r < P.nrays) e = Et[r];
            int cell = -1;
            if (r < P.nrays && e.base >= 0) {
                const int iy0 = e.base / P.sx, ix0 = e.base - iy0 * P.sx;
                cell = iy0 * P.ncx + ix0;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, cell);
            const int rank = __popc(peers & lt);
            if (cell >= 0) {
                const int pos = sh_counts[cell] + rank;
                E[pos] = e;
                inv[r] = pos;
            } else if (r < P.nrays) {
                inv[r] = -1;
            }
            __syncwarp();
            if (cell >= 0 && rank == 0) sh_counts[cell] += __popc(peers);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// convolution on a TILE x TILE output tile:
//   out[r][c] = sum_{a,b} taps[a][b] * Pb[(y0 + r + a) * Wp + x0 + c + b]
// taps = flipped PSF gives B, taps = PSF gives B^T (Section 2.2 operator).
// ---------------------------------------------------------------------------
template <typename T, int K, bool SH>
__device__ __forceinline__ void conv_tile(const T* __restrict__ Pb, int Wp, const T* __restrict__ taps,
                                          T (&acc)[TILE][TILE]) {
    constexpr int VW = Vec16<T>::n;
    constexpr int W = TILE + K - 1;
    constexpr int NVW = (W + VW - 1) / VW * VW;
    constexpr int KP = (K + 3) & ~3;
    const unsigned tap_a = smem_addr(taps);
    const unsigned src_a = SH ? smem_addr(Pb) : 0u;
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int c = 0; c < TILE; ++c) acc[r][c] = 0;
#pragma unroll
    for (int i = 0; i < TILE + K - 1; ++i) {
        T in[NVW];
#pragma unroll
        for (int v = 0; v < NVW; v += VW) {
            if (SH)
                lds_vec(src_a + (unsigned)((i * Wp + v) * sizeof(T)), in + v);
            else
                vload(Pb + i * Wp + v, in + v);
        }
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            const int a = i - r;
            if (a >= 0 && a < K) {
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    const T t = lds_one(tap_a + (unsigned)((a * KP + b) * sizeof(T)), T(0));
#pragma unroll
                    for (int c = 0; c < TILE; ++c) acc[r][c] = fma(t, in[c + b], acc[r][c]);
                }
            }
        }
    }
}

// runtime-K fallback
template <typename T>
__device__ __forceinline__ void conv_tile_rt(const T* __restrict__ Pb, int Wp, const T* __restrict__ taps,
                                             int K, int KP, T (&acc)[TILE][TILE]) {
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int c = 0; c < TILE; ++c) acc[r][c] = 0;
    for (int a = 0; a < K; ++a) {
        for (int b = 0; b < K; ++b) {
            const T t = taps[a * KP + b];
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const T* row = Pb + (r + a) * Wp + b;
#pragma unroll
                for (int c = 0; c < TILE; ++c) acc[r][c] = fma(t, row[c], acc[r][c]);
            }
        }
    }
}

template <typename T, int K, bool SH>
__device__ __forceinline__ void conv_any(const T* Pb, int Wp, const T* taps, int Krt, int KP,
                                         T (&acc)[TILE][TILE]) {
    if constexpr (K > 0) {
        conv_tile<T, K, SH>(Pb, Wp, taps, acc);
    } else {
        conv_tile_rt<T>(Pb, Wp, taps, Krt, KP, acc);
    }
}

// ---------------------------------------------------------------------------
// work-item state: pointers into shared memory (or the per-CTA global slab)
// ---------------------------------------------------------------------------
template <typename T>
struct Work {
    T* taps;      // [2][K][KP]: flipped PSF (B), PSF (B^T)
    T* swp;       // [plen] sqrt(W)
    T* rimg;      // [plen] image-space residual r = sqrt(W)(d - B L x)
    T* qimg;      // [plen] sqrt(W) B L p, later reused for u = B^T sqrt(W) r
    T* P1;        // [plen] padded conv input (L p)
    T* P2;        // [plen] padded conv input (sqrt(W) r)
    const Entry<T>* E;
    const int* inv;
    const int* cst;
    T* x;         // [ns]
    T* p;         // [ns]
    T* s;         // [ns]
    T* rreg;      // [nreg]
    T* qreg;      // [nreg]
};

// P1 <- L v on the tiles owned by this thread (Section 2.2: interpolation of
// the back-traced rays on the source grid, averaged over sub-pixels)
template <typename T>
__device__ __forceinline__ void apply_L(const Prob<T>& P, const Work<T>& w, const T* __restrict__ v) {
    for (int t = threadIdx.x; t < P.ntiles; t += blockDim.x) {
        const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            const int y = ty * TILE + r;
#pragma unroll
            for (int cc = 0; cc < TILE; ++cc) {
                const int x = tx * TILE + cc;
                if (y < P.ny && x < P.nx) {
                    const int j = y * P.nx + x;
                    T val = 0;
                    for (int a = 0; a < P.Np; ++a) {
                        const int e = w.inv[j * P.Np + a];
                        if (e >= 0) {
                            const Entry<T> en = w.E[e];
                            const T u = en.u, vv = en.v;
                            const T* s0 = v + en.base;
                            val += ((T)1 - vv) * (((T)1 - u) * s0[0] + u * s0[1]) +
                                   vv * (((T)1 - u) * s0[P.sx] + u * s0[P.sx + 1]);
                        }
                    }
                    w.P1[(y + P.hk) * P.Wp + x + P.hk] = val * P.invNp;
                }
            }
        }
    }
}

// (L^T u)_i for source pixel i: gather over the rays of the (up to) four
// cells that have i as a corner, in sorted (deterministic) order.
template <typename T>
__device__ __forceinline__ T apply_LT_at(const Prob<T>& P, const Work<T>& w, const T* __restrict__ U, int i,
                                         int ia, int ib) {
    T acc = 0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int iy0 = ib - dy;
        if (iy0 < 0 || iy0 > P.sy - 2) continue;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int ix0 = ia - dx;
            if (ix0 < 0 || ix0 > P.sx - 2) continue;
            const int cell = iy0 * P.ncx + ix0;
            const int k1 = w.cst[cell + 1];
            for (int k = w.cst[cell]; k < k1; ++k) {
                const Entry<T> en = w.E[k];
                const T wu = dx ? en.u : (T)1 - en.u;
                const T wv = dy ? en.v : (T)1 - en.v;
                acc += wu * wv * U[en.ppos];
            }
        }
    }
    (void)i;
    return acc * P.invNp;
}

// (H v) at row `row` of H (rows 0..ns-1, and ns..2ns-1 for Dy of the gradient)
template <typename T>
__device__ __forceinline__ T apply_H_row(const Prob<T>& P, const T* __restrict__ v, int row) {
    if (P.reg == 0) return v[row];
    if (P.reg == 2) {
        const int ib = row / P.sx, ia = row - ib * P.sx;
        T acc = (T)4 * v[row];
        if (ia > 0) acc -= v[row - 1];
        if (ia < P.sx - 1) acc -= v[row + 1];
        if (ib > 0) acc -= v[row - P.sx];
        if (ib < P.sy - 1) acc -= v[row + P.sx];
        return acc;
    }
    // gradient: Dx rows then Dy rows, zero beyond the grid
    if (row < P.ns) {
        const int ib = row / P.sx, ia = row - ib * P.sx;
        return (ia < P.sx - 1 ? v[row + 1] : (T)0) - v[row];
    }
    const int i = row - P.ns;
    const int ib = i / P.sx;
    return (ib < P.sy - 1 ? v[i + P.sx] : (T)0) - v[i];
}

// (H^T r)_i
template <typename T>
__device__ __forceinline__ T apply_HT_at(const Prob<T>& P, const T* __restrict__ r, int i, int ia, int ib) {
    if (P.reg == 0) return r[i];
    if (P.reg == 2) {  // symmetric
        T acc = (T)4 * r[i];
        if (ia > 0) acc -= r[i - 1];
        if (ia < P.sx - 1) acc -= r[i + 1];
        if (ib > 0) acc -= r[i - P.sx];
        if (ib < P.sy - 1) acc -= r[i + P.sx];
        return acc;
    }
    // Dx^T rx: rx[i-1] (if ia > 0) - rx[i];  Dy^T ry: ry[i-sx] (if ib > 0) - ry[i]
    const T* ry = r + P.ns;
    T acc = -r[i] - ry[i];
    if (ia > 0) acc += r[i - 1];
    if (ib > 0) acc += ry[i - P.sx];
    return acc;
}

// One convolution over all owned tiles with a mode-dependent epilogue (one
// inlined copy of the unrolled tile code per kernel):
//   CONV_Q   : dst = sqrt(W) * conv                 returns sum dst^2
//   CONV_RAW : dst = conv
//   CONV_RES : res = sqrt(W) d - sqrt(W) * conv; rimg = res; P2 = sqrt(W) res
//              returns sum res^2  (per-pixel terms in FP64)
enum : int { CONV_Q = 0, CONV_RAW = 1, CONV_RES = 2 };

template <typename T, int K, bool SH>
__device__ __noinline__ double conv_pass(const Prob<T>& P, const Work<T>& w, const T* __restrict__ src,
                                         const T* __restrict__ taps, T* __restrict__ dst,
                                         const T* __restrict__ bwp, int mode) {
    T ss = 0;
    double sd = 0;
    for (int t = threadIdx.x; t < P.ntiles; t += blockDim.x) {
        const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
        T acc[TILE][TILE];
        conv_any<T, K, SH>(src + (ty * TILE) * P.Wp + tx * TILE, P.Wp, taps, P.K, P.kp, acc);
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            const int pp = (ty * TILE + r + P.hk) * P.Wp + tx * TILE + P.hk;
#pragma unroll
            for (int cc = 0; cc < TILE; ++cc) {
                if (mode == CONV_Q) {
                    const T q = w.swp[pp + cc] * acc[r][cc];
                    dst[pp + cc] = q;
                    ss = fma(q, q, ss);
                } else if (mode == CONV_RAW) {
                    dst[pp + cc] = acc[r][cc];
                } else {
                    const T sw = w.swp[pp + cc];
                    const T res = bwp[pp + cc] - sw * acc[r][cc];
                    w.rimg[pp + cc] = res;
                    w.P2[pp + cc] = sw * res;
                    sd += (double)res * (double)res;
                }
            }
        }
    }
    return (double)ss + sd;
}

// s = A~^T r = L^T B^T (sqrt(W) r_img) + sqrt(lam) H^T r_reg, given
// P2 = sqrt(W) r_img already in place.  Returns ||s||^2 (block-reduced).
template <typename T, int K, bool SH>
__device__ __forceinline__ double normal_residual(const Prob<T>& P, const Work<T>& w, T sl, bool with_reg,
                                                  double* red, int& which) {
    __syncthreads();  // P2 complete
    conv_pass<T, K, SH>(P, w, w.P2, w.taps + P.K * P.kp, w.qimg, nullptr, CONV_RAW);
    __syncthreads();  // u complete
    T ss = 0;  // per-thread partial in T, cross-thread sum in FP64
    for (int i = threadIdx.x; i < P.ns; i += blockDim.x) {
        const int ib = i / P.sx, ia = i - ib * P.sx;
        T v = apply_LT_at(P, w, w.qimg, i, ia, ib);
        if (with_reg) v += sl * apply_HT_at(P, w.rreg, i, ia, ib);
        w.s[i] = v;
        ss = fma(v, v, ss);
    }
    const double r = block_sum((double)ss, red, which);
    which ^= 1;
    return r;
}

// r_img = sqrt(W)(d - B L x), r_reg = -sqrt(lam) H x; returns chi2 = ||r_img||^2.
// Leaves P2 = sqrt(W) r_img (no trailing barrier).
template <typename T, int K, bool SH>
__device__ __forceinline__ double true_residual(const Prob<T>& P, const Work<T>& w, const T* __restrict__ bwp,
                                                T sl, double* red, int& which) {
    apply_L(P, w, w.x);
    for (int i = threadIdx.x; i < P.nreg; i += blockDim.x) w.rreg[i] = -sl * apply_H_row(P, w.x, i);
    __syncthreads();
    const double chi = conv_pass<T, K, SH>(P, w, w.P1, w.taps, nullptr, bwp, CONV_RES);
    const double c = block_sum(chi, red, which);
    which ^= 1;
    return c;
}

// ---------------------------------------------------------------------------
// k_cgls: persistent CTAs, one (candidate, lambda) item at a time
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t align_up(size_t v, size_t a) {
    return (v + a - 1) / a * a;
}

// Shared-memory footprint of the SMEM-resident layout of one problem.
template <typename T>
__host__ __device__ inline size_t smem_bytes(const Prob<T>& P, bool big) {
    size_t o = 0;
    o += align_up<T>(sizeof(T) * 2 * P.K * P.kp, 16);  // taps
    o += 2 * 33 * sizeof(double) + 16;                  // reductions + item slot
    if (!big) {
        o += 5 * align_up<T>(sizeof(T) * P.plen, 16);                  // swp rimg qimg P1 P2
        o += align_up<T>(sizeof(Entry<T>) * (size_t)P.nrays, 16);      // E
        o += align_up<T>(sizeof(int) * (size_t)P.nrays, 16);           // inv
        o += align_up<T>(sizeof(int) * (size_t)(P.ncells + 1), 16);    // cst
        o += 3 * align_up<T>(sizeof(T) * P.ns, 16);                    // x p s
        o += 2 * align_up<T>(sizeof(T) * P.nreg, 16);                  // rreg qreg
    }
    return o;
}

template <typename T>
__host__ __device__ inline size_t slab_elems(const Prob<T>& P) {
    // BIG variant: rimg qimg P1 P2 + x p s + rreg qreg in global memory
    return 4 * align_up<T>(P.plen, 4) + 3 * align_up<T>(P.ns, 4) + 2 * align_up<T>(P.nreg, 4);
}

template <typename T, int K, bool BIG>
__global__ void __launch_bounds__(NTHREADS, 1) k_cgls(CglsArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, bs = blockDim.x;
    int last_c = -1, last_prob = -1;
    Work<T> w;
    int which = 0;

    while (true) {
        unsigned char* sp = smem;
        const Prob<T>* Pp;
        // --- fetch the next item
        int* slot = reinterpret_cast<int*>(smem + 0);
        // carve: item slot (16 B) first so it never moves
        sp += 16;
        __syncthreads();
        if (tid == 0) slot[0] = atomicAdd(A.counter, 1);
        __syncthreads();
        const int it_idx = slot[0];
        if (it_idx >= A.n_items) break;
        const int packed = A.items[it_idx];
        const int c = packed / MAX_LAM, k = packed - c * MAX_LAM;
        const int pi = A.cand_prob[c];
        Pp = A.probs + pi;
        const Prob<T> P = *Pp;

        double* red = reinterpret_cast<double*>(sp);
        sp += 2 * 33 * sizeof(double);
        w.taps = reinterpret_cast<T*>(sp);
        sp += align_up<T>(sizeof(T) * 2 * P.K * P.kp, 16);

        const CandScratch<T>& cs = A.cs;
        const T* g_swp = cs.swp + (long long)c * cs.sPad;
        const T* g_bwp = cs.bwp + (long long)c * cs.sPad;
        const Entry<T>* g_E = cs.E + (long long)c * cs.sE;
        const int* g_inv = cs.inv + (long long)c * cs.sInv;
        const int* g_cst = cs.cst + (long long)c * cs.sCst;

        if constexpr (!BIG) {
            const size_t pl = align_up<T>(sizeof(T) * P.plen, 16);
            w.swp = reinterpret_cast<T*>(sp); sp += pl;
            w.rimg = reinterpret_cast<T*>(sp); sp += pl;
            w.qimg = reinterpret_cast<T*>(sp); sp += pl;
            w.P1 = reinterpret_cast<T*>(sp); sp += pl;
            w.P2 = reinterpret_cast<T*>(sp); sp += pl;
            Entry<T>* sE = reinterpret_cast<Entry<T>*>(sp);
            sp += align_up<T>(sizeof(Entry<T>) * (size_t)P.nrays, 16);
            int* sInv = reinterpret_cast<int*>(sp);
            sp += align_up<T>(sizeof(int) * (size_t)P.nrays, 16);
            int* sCst = reinterpret_cast<int*>(sp);
            sp += align_up<T>(sizeof(int) * (size_t)(P.ncells + 1), 16);
            const size_t ps = align_up<T>(sizeof(T) * P.ns, 16);
            const size_t pr = align_up<T>(sizeof(T) * P.nreg, 16);
            w.x = reinterpret_cast<T*>(sp); sp += ps;
            w.p = reinterpret_cast<T*>(sp); sp += ps;
            w.s = reinterpret_cast<T*>(sp); sp += ps;
            w.rreg = reinterpret_cast<T*>(sp); sp += pr;
            w.qreg = reinterpret_cast<T*>(sp); sp += pr;
            w.E = sE;
            w.inv = sInv;
            w.cst = sCst;
            if (c != last_c) {
                // stage the candidate's lens operator and weights in shared memory
                const int ne = A.cs.nent[c];
                for (int i = tid; i < ne; i += bs) sE[i] = g_E[i];
                for (int i = tid; i < P.nrays; i += bs) sInv[i] = g_inv[i];
                for (int i = tid; i <= P.ncells; i += bs) sCst[i] = g_cst[i];
                for (int i = tid; i < P.plen; i += bs) w.swp[i] = g_swp[i];
            }
        } else {
            T* slab = A.slab + (long long)blockIdx.x * A.slab_stride;
            const size_t pl = align_up<T>(P.plen, 4);
            w.rimg = slab; slab += pl;
            w.qimg = slab; slab += pl;
            w.P1 = slab; slab += pl;
            w.P2 = slab; slab += pl;
            w.x = slab; slab += align_up<T>(P.ns, 4);
            w.p = slab; slab += align_up<T>(P.ns, 4);
            w.s = slab; slab += align_up<T>(P.ns, 4);
            w.rreg = slab; slab += align_up<T>(P.nreg, 4);
            w.qreg = slab; slab += align_up<T>(P.nreg, 4);
            w.swp = const_cast<T*>(g_swp);
            w.E = g_E;
            w.inv = g_inv;
            w.cst = g_cst;
        }
        if (pi != last_prob || c != last_c) {
            // taps: [0] flipped PSF for B, [1] PSF for B^T; rows padded to kp
            for (int i = tid; i < 2 * P.K * P.kp; i += bs) {
                const int h = i / (P.K * P.kp), rem = i - h * P.K * P.kp;
                const int a = rem / P.kp, b = rem - a * P.kp;
                T v = 0;
                if (b < P.K) v = h == 0 ? P.psf[(P.K - 1 - a) * P.K + (P.K - 1 - b)] : P.psf[a * P.K + b];
                w.taps[i] = v;
            }
        }
        last_c = c;
        last_prob = pi;
        for (int i = tid; i < P.plen; i += bs) {
            w.P1[i] = 0;
            w.P2[i] = 0;
        }
        __syncthreads();

        const int cstat = A.cs.cstat[c];
        const long long ok = (long long)c * A.max_lam + k;
        T* X = A.X + ok * A.max_ns;
        if (cstat & (ST_BADPARAM | ST_EMPTY)) {
            for (int i = tid; i < P.ns; i += bs) X[i] = 0;
            if (tid == 0) {
                A.chi2[ok] = (cstat & ST_BADPARAM) ? __longlong_as_double(0x7ff0000000000000LL) : 0.0;
                A.reg[ok] = 0.0;
                A.iters[ok] = 0;
                if (A.relres) A.relres[ok] = 0.0;
                if (A.istat) A.istat[ok] = cstat;
            }
            continue;
        }

        const double lam = A.lambdas[(long long)c * A.max_lam + k];
        const T sl = (T)sqrt(lam);
        const int maxit = A.maxit > 0 ? A.maxit : 10 * P.ns;
        const int rep = A.replace_every > 0 ? A.replace_every : 50;

        // ||rhs|| = ||L^T B^T sqrt(W) (sqrt(W) d)||
        for (int t = tid; t < P.ntiles; t += bs) {
            const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int pp = (ty * TILE + r + P.hk) * P.Wp + tx * TILE + P.hk;
#pragma unroll
                for (int cc = 0; cc < TILE; ++cc) w.P2[pp + cc] = w.swp[pp + cc] * g_bwp[pp + cc];
            }
        }
        const double rhs2 = normal_residual<T, K, !BIG>(P, w, sl, false, red, which);
        const double rhsn = sqrt(rhs2);

        double gam;
        if (A.warm_x) {
            const T* x0 = A.warm_x + ok * A.max_ns;
            for (int i = tid; i < P.ns; i += bs) w.x[i] = x0[i];
            __syncthreads();
            true_residual<T, K, !BIG>(P, w, g_bwp, sl, red, which);
            gam = normal_residual<T, K, !BIG>(P, w, sl, true, red, which);
        } else {
            // x = 0: r_img = sqrt(W) d, r_reg = 0, s = rhs (already in w.s)
            for (int i = tid; i < P.ns; i += bs) w.x[i] = 0;
            for (int i = tid; i < P.nreg; i += bs) w.rreg[i] = 0;
            for (int i = tid; i < P.plen; i += bs) w.rimg[i] = g_bwp[i];
            gam = rhs2;
        }
        for (int i = tid; i < P.ns; i += bs) w.p[i] = w.s[i];
        __syncthreads();

        int status = 0, it = 0;
        double best = (rhsn > 0) ? sqrt(gam) / rhsn : 0.0;
        int best_it = 0;
        const int stag_window = max(2000, P.ns);
        for (it = 0;; ++it) {
            if (!isfinite(gam)) {
                status |= ST_BREAK;
                break;
            }
            const double rel = (rhsn > 0) ? sqrt(gam) / rhsn : 0.0;
            if (!(rel > A.tol)) break;  // converged (or rhs = 0)
            if (it >= maxit) {
                status |= ST_MAXIT;
                break;
            }
            if (rel < 0.5 * best) {
                best = rel;
                best_it = it;
            } else if (it - best_it > stag_window) {
                status |= ST_STAG;
                break;
            }
            // q = A~ p: image part sqrt(W) B L p, regulariser part sqrt(lam) H p
            apply_L(P, w, w.p);
            T dqr = 0;
            for (int i = tid; i < P.nreg; i += bs) {
                const T q = sl * apply_H_row(P, w.p, i);
                w.qreg[i] = q;
                dqr = fma(q, q, dqr);
            }
            __syncthreads();
            const double dq = (double)dqr + conv_pass<T, K, !BIG>(P, w, w.P1, w.taps, w.qimg, nullptr, CONV_Q);
            const double delta = block_sum(dq, red, which);
            which ^= 1;
            if (!(delta > 0.0) || !isfinite(delta)) {
                status |= ST_BREAK;
                break;
            }
            const double alpha = gam / delta;
            const T a = (T)alpha;
            for (int i = tid; i < P.ns; i += bs) w.x[i] = fma(a, w.p[i], w.x[i]);
            for (int i = tid; i < P.nreg; i += bs) w.rreg[i] = fma(-a, w.qreg[i], w.rreg[i]);
            const bool replace = ((it + 1) % rep) == 0;
            if (!replace) {
                for (int t = tid; t < P.ntiles; t += bs) {
                    const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
#pragma unroll
                    for (int r = 0; r < TILE; ++r) {
                        const int pp = (ty * TILE + r + P.hk) * P.Wp + tx * TILE + P.hk;
#pragma unroll
                        for (int cc = 0; cc < TILE; ++cc) {
                            const T rv = fma(-a, w.qimg[pp + cc], w.rimg[pp + cc]);
                            w.rimg[pp + cc] = rv;
                            w.P2[pp + cc] = w.swp[pp + cc] * rv;
                        }
                    }
                }
            } else {
                __syncthreads();  // x complete
                true_residual<T, K, !BIG>(P, w, g_bwp, sl, red, which);
            }
            const double gnew = normal_residual<T, K, !BIG>(P, w, sl, true, red, which);
            const double beta = gnew / gam;
            gam = gnew;
            const T bt = (T)beta;
            for (int i = tid; i < P.ns; i += bs) w.p[i] = fma(bt, w.p[i], w.s[i]);
            __syncthreads();
        }

        // outputs: chi2 from the true residual, ||H x||^2, true relative residual
        __syncthreads();
        const double chi2 = true_residual<T, K, !BIG>(P, w, g_bwp, sl, red, which);
        double hx = 0;
        for (int i = tid; i < P.nreg; i += bs) {
            const double v = (double)apply_H_row(P, w.x, i);
            hx += v * v;
        }
        const double reg2 = block_sum(hx, red, which);
        which ^= 1;
        const double tr = normal_residual<T, K, !BIG>(P, w, sl, true, red, which);
        for (int i = tid; i < P.ns; i += bs) X[i] = w.x[i];
        if (tid == 0) {
            A.chi2[ok] = chi2;
            A.reg[ok] = reg2;
            A.iters[ok] = it;
            if (A.relres) A.relres[ok] = rhsn > 0 ? sqrt(tr) / rhsn : 0.0;
            if (A.istat) A.istat[ok] = status | cstat;
        }
    }
}

// ---------------------------------------------------------------------------
// k_finalize: L-curve corner per candidate (Section 2.6), status, s_out
// ---------------------------------------------------------------------------
__device__ inline int lcurve_corner_dev(const double* chi2, const double* reg, int n, double* kappa,
                                        int* flat) {
    double x[MAX_LAM], y[MAX_LAM], t[MAX_LAM], Mx[MAX_LAM], My[MAX_LAM], cp[MAX_LAM];
    int idx[MAX_LAM];
    for (int i = 0; i < n; ++i) kappa[i] = 0.0;
    *flat = 1;
    if (n < 3) return n > 0 ? (n - 1) / 2 : 0;
    double px[MAX_LAM], py[MAX_LAM];
    for (int i = 0; i < n; ++i) {
        px[i] = log10(fmax(reg[i], 1e-300));
        py[i] = log10(fmax(chi2[i], 1e-300));
    }
    double total = 0.0;
    for (int i = 1; i < n; ++i) total += hypot(px[i] - px[i - 1], py[i] - py[i - 1]);
    int m = 0;
    idx[m] = 0;
    x[m] = px[0];
    y[m] = py[0];
    t[m] = 0.0;
    ++m;
    for (int i = 1; i < n; ++i) {
        const double st = hypot(px[i] - px[i - 1], py[i] - py[i - 1]);
        if (total > 0.0 && st > 1e-12 * total) {
            // chord length between consecutive kept points
            const double h = hypot(px[i] - x[m - 1], py[i] - y[m - 1]);
            idx[m] = i;
            x[m] = px[i];
            y[m] = py[i];
            t[m] = t[m - 1] + h;
            ++m;
        }
    }
    if (m < 3) return (n - 1) / 2;
    // natural cubic spline second derivatives by the tridiagonal (Thomas) solve
    for (int pass = 0; pass < 2; ++pass) {
        const double* f = pass ? y : x;
        double* M = pass ? My : Mx;
        M[0] = 0.0;
        M[m - 1] = 0.0;
        // forward sweep on rows 1..m-2
        double cprev = 0.0, rprev = 0.0;
        for (int i = 1; i <= m - 2; ++i) {
            const double h0 = t[i] - t[i - 1], h1 = t[i + 1] - t[i];
            const double a = h0, b = 2.0 * (h0 + h1), cc = h1;
            const double r = 6.0 * ((f[i + 1] - f[i]) / h1 - (f[i] - f[i - 1]) / h0);
            double denom = b, rr = r;
            if (i > 1) {
                denom = b - a * cprev;
                rr = r - a * rprev;
            }
            cp[i] = cc / denom;
            const double rn = rr / denom;
            cprev = cp[i];
            rprev = rn;
            M[i] = rn;  // temporarily the modified rhs
        }
        for (int i = m - 3; i >= 1; --i) M[i] -= cp[i] * M[i + 1];
    }
    double kmax = 0.0;
    int arg = -1;
    for (int i = 1; i < m - 1; ++i) {
        const double h = t[i + 1] - t[i];
        const double x1 = (x[i + 1] - x[i]) / h - h * (2.0 * Mx[i] + Mx[i + 1]) / 6.0;
        const double y1 = (y[i + 1] - y[i]) / h - h * (2.0 * My[i] + My[i + 1]) / 6.0;
        const double x2 = Mx[i], y2 = My[i];
        const double den = pow(x1 * x1 + y1 * y1, 1.5);
        double k = fabs(x1 * y2 - y1 * x2) / den;
        if (!isfinite(k)) k = 0.0;  // tangent vanishes: curvature undefined
        kappa[idx[i]] = k;
        if (k > kmax) {
            kmax = k;
            arg = idx[i];
        }
    }
    if (arg < 0 || !(kmax * t[m - 1] > 1e-9)) return (n - 1) / 2;
    *flat = 0;
    return arg;
}

template <typename T>
__global__ void k_finalize(int cand0, int n_cand, int max_lam, int max_ns, const int* __restrict__ n_lam,
                           const int* __restrict__ cand_prob, const Prob<T>* __restrict__ probs,
                           const double* __restrict__ chi2, const double* __restrict__ reg,
                           const int* __restrict__ istat, const int* __restrict__ cstat, const T* __restrict__ X,
                           int* corner, double* kappa, T* s_out, int* status) {
    const int c = cand0 + blockIdx.x;
    if (c >= cand0 + n_cand) return;
    __shared__ int s_corner;
    if (threadIdx.x == 0) {
        const int n = n_lam[c];
        double kap[MAX_LAM];
        int flat = 0;
        const int cn = lcurve_corner_dev(chi2 + (long long)c * max_lam, reg + (long long)c * max_lam, n, kap,
                                         &flat);
        if (kappa)
            for (int i = 0; i < n; ++i) kappa[(long long)c * max_lam + i] = kap[i];
        int st = cstat[c] | (flat ? ST_FLAT : 0);
        for (int i = 0; i < n; ++i) st |= istat[(long long)c * max_lam + i];
        corner[c] = cn;
        status[c] = st;
        s_corner = cn;
    }
    __syncthreads();
    if (s_out) {
        const int ns = probs[cand_prob[c]].ns;
        const T* src = X + ((long long)c * max_lam + s_corner) * max_ns;
        for (int i = threadIdx.x; i < ns; i += blockDim.x) s_out[(long long)c * max_ns + i] = src[i];
    }
}

// standalone L-curve over device arrays (one thread per candidate)
template <int UNUSED = 0>
__global__ void k_lcurve(const double* __restrict__ chi2, const double* __restrict__ reg,
                         const int* __restrict__ n_lam, int n_cand, int max_lam, int* corner, double* kappa,
                         int* flags) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand) return;
    double kap[MAX_LAM];
    int flat = 0;
    const int n = min(n_lam[c], MAX_LAM);
    const int cn = lcurve_corner_dev(chi2 + (long long)c * max_lam, reg + (long long)c * max_lam, n, kap, &flat);
    corner[c] = cn;
    if (kappa)
        for (int i = 0; i < n; ++i) kappa[(long long)c * max_lam + i] = kap[i];
    if (flags) flags[c] = flat ? ST_FLAT : 0;
}

// ---------------------------------------------------------------------------
// k_forward: model = B L s and chi2 for a batch of sources at one lens
// (candidate scratch of index 0).  One CTA per source (grid-stride).
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(NTHREADS, 1) k_forward(const Prob<T>* __restrict__ probs, CandScratch<T> cs,
                                                         const T* __restrict__ S, int n_src, T* model,
                                                         double* chi2, T* slab, long long slab_stride,
                                                         int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob<T> P = probs[0];
    unsigned char* sp = smem;
    double* red = reinterpret_cast<double*>(sp);
    sp += 2 * 33 * sizeof(double) + 16;
    Work<T> w;
    w.taps = reinterpret_cast<T*>(sp);
    sp += align_up<T>(sizeof(T) * 2 * P.K * P.kp, 16);
    w.P1 = slab + (long long)blockIdx.x * slab_stride;
    w.swp = cs.swp;
    w.E = cs.E;
    w.inv = cs.inv;
    w.cst = cs.cst;
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * P.K * P.kp; i += blockDim.x) {
        const int h = i / (P.K * P.kp), rem = i - h * P.K * P.kp;
        const int a = rem / P.kp, b = rem - a * P.kp;
        T v = 0;
        if (b < P.K) v = h == 0 ? P.psf[(P.K - 1 - a) * P.K + (P.K - 1 - b)] : P.psf[a * P.K + b];
        w.taps[i] = v;
    }
    for (int i = tid; i < P.plen; i += blockDim.x) w.P1[i] = 0;
    if (blockIdx.x == 0 && tid == 0 && status) status[0] = cs.cstat[0];
    int which = 0;
    const bool bad = (cs.cstat[0] & ST_BADPARAM) != 0;
    for (int k = blockIdx.x; k < n_src; k += gridDim.x) {
        __syncthreads();
        if (bad) {
            if (tid == 0) chi2[k] = __longlong_as_double(0x7ff0000000000000LL);
            continue;
        }
        apply_L(P, w, S + (long long)k * P.ns);
        __syncthreads();
        double chi = 0;
        for (int t = tid; t < P.ntiles; t += blockDim.x) {
            const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
            T acc[TILE][TILE];
            conv_any<T, K, false>(w.P1 + (ty * TILE) * P.Wp + tx * TILE, P.Wp, w.taps, P.K, P.kp, acc);
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int y = ty * TILE + r;
                const int pp = (y + P.hk) * P.Wp + tx * TILE + P.hk;
#pragma unroll
                for (int cc = 0; cc < TILE; ++cc) {
                    const int x = tx * TILE + cc;
                    const T res = cs.bwp[pp + cc] - cs.swp[pp + cc] * acc[r][cc];
                    chi += (double)res * (double)res;
                    if (model && y < P.ny && x < P.nx) model[(long long)k * P.npix + y * P.nx + x] = acc[r][cc];
                }
            }
        }
        const double cval = block_sum(chi, red, which);
        which ^= 1;
        if (tid == 0) chi2[k] = cval;
    }
}

}  // namespace mirage
