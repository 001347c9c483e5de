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
//                zero-padded convolutions on 4x4 register tiles.  FP32
//                inner solves sit inside an FP64 residual refinement.
//   k_finalize   L-curve corner (Section 2.6) per candidate, status, s_out.
//   k_forward    B L s and Eq. chi2 for a batch of sources at one lens.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"
#include "fftconv.cuh"
#include "interp.cuh"
#include "lcurve.cuh"
#include "lens.cuh"
#include "reg.cuh"

namespace mirage {

constexpr int TILE = 4;        // each thread owns TILE x TILE image pixels in the convolutions
constexpr int NTHREADS = 256;  // CTA size of the item kernels
// MAX_LAM (longest lambda grid of one candidate) comes with lcurve.cuh

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
    int nx, ny, npix, sx, sy, ns, nreg, K, hk, n_sub, Np, nrays, ncx, ncells, reg, interp;
    int Wp, Hp, plen, tiles_x, tiles_y, ntiles, kp, xoff;  // padded layout, tap row pitch, left pad
    int fft_m, fft_log;  // FFT convolution grid side and its log2 (0: direct convolution)
    double pix, cx, cy, sub0, subd, c0x, c0y, hx, hy;  // ray-trace geometry (always FP64)
    T invNp;
    const T* d;
    const T* sigma;
    const uint8_t* mask;
    const T* psf;
};

// Per-candidate scratch written by k_raytrace (strides in elements).
template <typename T>
struct CandScratch {
    Entry<T>* E;      // [n_cand][sE]  sorted mapped rays (weights in T)
    Entry<double>* E64;   // [n_cand][sE] the same rays with FP64 weights (aliases E when T = double)
    Entry<double>* Etmp;  // [n_cand][sE] rays in ray order (build only)
    int* inv;         // [n_cand][sInv] ray -> sorted position, -1 unmapped
    int* cst;         // [n_cand][sCst] cell start offsets (ncells + 1)
    T* swp;           // [n_cand][sPad] m / sigma in padded layout
    T* dpad;          // [n_cand][sPad] observed image in padded layout
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
    const int* items;       // [n_items] packed chains (c * MAX_LAM + k_first) * MAX_LAM + k_last
    int n_items;
    int* counter;           // queue head
    double tol;
    double eta;             // FP32 contexts: inner-solve reduction target of the refinement
    int maxit;              // <= 0: 10 * ns
    int replace_every;
    int max_lam, max_ns;
    const T* warm_x;        // nullable [n_cand][max_lam][max_ns]
    CandScratch<T> cs;
    void* slab;             // per-CTA global work buffers (FP64 refinement; all buffers if BIG)
    long long slab_stride;  // bytes
    T* X;                   // [n_cand][max_lam][max_ns]
    double* chi2;           // [n_cand][max_lam]
    double* reg;
    int* iters;
    double* relres;
    int* istat;
    unsigned long long* phase_clk;  // nullable [8]: per-phase SM clock totals (instrumented runs)
    const float2* spec32;   // PSF spectra of the FFT problems, [n_probs][spec_stride] (FP32 contexts)
    const double2* spec64;  // the same in FP64
    long long spec_stride;  // elements per problem
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// (m_atan, m_atanh, m_sqrt, m_floor: lens.cuh)

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

// Block sum of non-negative terms delivered to thread 0 only (FP64 across
// warps); other threads get 0.  The caller lets thread 0 derive its
// scalars, then synchronises.  FP32 terms are summed within a warp by a
// plain FP32 butterfly: sums of non-negative terms have no cancellation, so
// this keeps ~5 2^-24 relative accuracy, ample for the inner solves' CG
// coefficients (the refinement's sums are FP64).
template <typename T>
__device__ __forceinline__ double block_sum_to0(T v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double wv;
    if constexpr (sizeof(T) == 4) {
        float f = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        wv = (double)f;
    } else {
        wv = warp_sum((double)v);
    }
    if (lane == 0) red[warp] = wv;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// Scalars of the inner CGLS, written by thread 0 and read by all threads
// after a barrier.
struct CgCtl {
    double gam, g0, best;
    int best_it, it, total_it, stop, brk;
    float a_f, b_f;
    double a_d, b_d;
};
static_assert(sizeof(CgCtl) <= 128, "CG control block must fit its reserved shared-memory slot");

// ---------------------------------------------------------------------------
// lens model
// ---------------------------------------------------------------------------
// (LensT, make_lens, trace_ray: lens.cuh)

// ---------------------------------------------------------------------------
// Ray trace of one candidate, in two parts shared by the kernels below:
//   rt_trace_pixels : trace the rays of image pixels [j0, j1) (this CTA's
//                     threads), write them in ray order, sqrt(W) and the
//                     padded data, and count rays per cell into `counts`
//                     and active pixels into `active` (shared or global);
//   rt_place        : scan the cell counts and place the rays sorted by
//                     cell, stable within a cell (one warp, in ray order).
// Rays are traced in FP64 whatever T is: the refinement residual uses these
// weights, and FP32-rounded weights would perturb the operator by ~1e-7,
// which the conditioning of small-lambda systems amplifies.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void rt_trace_pixels(const Prob<T>& P, const LensT<double>& L, const CandScratch<T>& cs,
                                                int c, int j0, int j1, int* counts, int* active) {
    Entry<double>* Et = cs.Etmp + (long long)c * cs.sE;
    T* swp = cs.swp + (long long)c * cs.sPad;
    T* dpad = cs.dpad + (long long)c * cs.sPad;
    const double half_x = 0.5 * (double)(P.nx - 1), half_y = 0.5 * (double)(P.ny - 1);
    const double fxmax = (double)(P.sx - 1), fymax = (double)(P.sy - 1);
    int my_active = 0;
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
        const int x = j % P.nx, y = j / P.nx;
        const double tx = P.cx + ((double)x - half_x) * P.pix;
        const double ty = P.cy + ((double)y - half_y) * P.pix;
        const int pp = (y + P.hk) * P.Wp + x + P.xoff;
        bool any = false;
        for (int a = 0; a < P.Np; ++a) {
            const int ax = a % P.n_sub, ay = a / P.n_sub;
            double bx, by;
            trace_ray(L, tx + P.sub0 + (double)ax * P.subd, ty + P.sub0 + (double)ay * P.subd, bx, by);
            const double fx = (bx - P.c0x) / P.hx;
            const double fy = (by - P.c0y) / P.hy;
            const bool m = (fx >= 0.0) && (fx <= fxmax) && (fy >= 0.0) && (fy <= fymax);
            Entry<double> e;
            e.ppos = pp;
            if (m) {
                const int ix0 = min((int)m_floor(fx), P.sx - 2);
                const int iy0 = min((int)m_floor(fy), P.sy - 2);
                e.base = iy0 * P.sx + ix0;
                e.u = fx - (double)ix0;
                e.v = fy - (double)iy0;
                if (P.interp == 1) {  // nearest centre: the one-hot bilinear weights
                    e.u = e.u >= 0.5 ? 1.0 : 0.0;
                    e.v = e.v >= 0.5 ? 1.0 : 0.0;
                }
                atomicAdd(&counts[iy0 * P.ncx + ix0], 1);
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
        dpad[pp] = P.d[j];
        my_active += (w != (T)0);
    }
    if (my_active) atomicAdd(active, my_active);
}

// sh_counts: [ncells] shared memory holding the cell counts on entry;
// s_chunk: [NTHREADS] shared scratch; active: the candidate's active pixels
template <typename T>
__device__ __forceinline__ void rt_place(const Prob<T>& P, const CandScratch<T>& cs, int c, int* sh_counts,
                                         int* s_chunk, int active, bool place = true) {
    Entry<T>* E = cs.E + (long long)c * cs.sE;
    Entry<double>* E64 = cs.E64 + (long long)c * cs.sE;
    const Entry<double>* Et = cs.Etmp + (long long)c * cs.sE;
    int* inv = cs.inv + (long long)c * cs.sInv;
    int* cst = cs.cst + (long long)c * cs.sCst;
    const int tid = threadIdx.x, bs = blockDim.x;

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
        cs.cstat[c] = (active > 0) ? 0 : ST_EMPTY;
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
    if (!place) return;

    // pass 2: one warp places the rays in ray order (stable within a cell),
    // eight 32-ray batches at a time with the next eight already loading
    if (tid < 32) {
        const int lane = tid;
        const unsigned lt = (1u << lane) - 1u;
        constexpr int G = 8;
        Entry<double> nxt[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int r = q * 32 + lane;
            nxt[q].base = -1;
            if (r < P.nrays) nxt[q] = Et[r];
        }
        for (int g0 = 0; g0 < P.nrays; g0 += 32 * G) {
            Entry<double> cur[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                cur[q] = nxt[q];
                const int r = g0 + (G + q) * 32 + lane;
                nxt[q].base = -1;
                if (r < P.nrays) nxt[q] = Et[r];
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int r = g0 + q * 32 + lane;
                const Entry<double>& e = cur[q];
                int cell = -1;
                if (r < P.nrays && e.base >= 0) {
                    const int iy0 = e.base / P.sx, ix0 = e.base - iy0 * P.sx;
                    cell = iy0 * P.ncx + ix0;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, cell);
                const int rank = __popc(peers & lt);
                if (cell >= 0) {
                    const int pos = sh_counts[cell] + rank;
                    E64[pos] = e;
                    if ((void*)E != (void*)E64) {
                        Entry<T> et;
                        et.ppos = e.ppos;
                        et.base = e.base;
                        et.u = (T)e.u;
                        et.v = (T)e.v;
                        E[pos] = et;
                    }
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
}

// sets the outputs of a candidate whose lens parameters are invalid
template <typename T>
__device__ __forceinline__ void rt_bad(const Prob<T>& P, const CandScratch<T>& cs, int c) {
    int* inv = cs.inv + (long long)c * cs.sInv;
    int* cst = cs.cst + (long long)c * cs.sCst;
    for (int r = threadIdx.x; r < P.nrays; r += blockDim.x) inv[r] = -1;
    for (int i = threadIdx.x; i <= P.ncells; i += blockDim.x) cst[i] = 0;
    if (threadIdx.x == 0) {
        cs.nent[c] = 0;
        cs.cstat[c] = ST_BADPARAM;
    }
}

// ---------------------------------------------------------------------------
// k_raytrace: one CTA per candidate (trace, count, scan, place)
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
    T* swp = cs.swp + (long long)c * cs.sPad;
    T* dpad = cs.dpad + (long long)c * cs.sPad;
    const int tid = threadIdx.x, bs = blockDim.x;
    const LensT<double> L = make_lens<double>(lens + 7LL * c);

    for (int i = tid; i < P.plen; i += bs) {
        swp[i] = 0;
        dpad[i] = 0;
    }
    for (int i = tid; i < P.ncells; i += bs) sh_counts[i] = 0;
    if (tid == 0) s_active = 0;
    __syncthreads();
    if (L.bad) {
        rt_bad(P, cs, c);
        return;
    }
    rt_trace_pixels(P, L, cs, c, 0, P.npix, sh_counts, &s_active);
    __syncthreads();
    rt_place(P, cs, c, sh_counts, s_chunk, s_active);
}

// ---------------------------------------------------------------------------
// Split ray trace for few candidates with many rays (the forward batch and
// other small calls on large images): k_rt_trace spreads the rays of each
// candidate over blockIdx.x chunks of `chunk` pixels, counting into the
// candidate's cell-start array and its status word (both zeroed, with sqrt(W)
// and the padded data, by the caller); k_rt_place then scans and places
// them, one CTA per candidate.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rt_trace(const Prob<T>* __restrict__ probs,
                                                       const int* __restrict__ cand_prob,
                                                       const double* __restrict__ lens, int cand0, int chunk,
                                                       CandScratch<T> cs) {
    const int c = cand0 + blockIdx.y;
    const Prob<T>& P = probs[cand_prob[c]];
    const LensT<double> L = make_lens<double>(lens + 7LL * c);
    if (L.bad) return;
    const int j0 = blockIdx.x * chunk, j1 = min(j0 + chunk, P.npix);
    if (j0 >= j1) return;
    rt_trace_pixels(P, L, cs, c, j0, j1, cs.cst + (long long)c * cs.sCst, cs.cstat + c);
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rt_place(const Prob<T>* __restrict__ probs,
                                                       const int* __restrict__ cand_prob,
                                                       const double* __restrict__ lens, int cand0,
                                                       CandScratch<T> cs) {
    const int c = cand0 + blockIdx.x;
    const Prob<T>& P = probs[cand_prob[c]];
    extern __shared__ int sh_counts[];
    __shared__ int s_chunk[NTHREADS];
    const LensT<double> L = make_lens<double>(lens + 7LL * c);
    if (L.bad) {
        rt_bad(P, cs, c);
        return;
    }
    const int* cnt = cs.cst + (long long)c * cs.sCst;
    for (int i = threadIdx.x; i < P.ncells; i += blockDim.x) sh_counts[i] = cnt[i];
    const int active = cs.cstat[c];
    __syncthreads();
    // one ray per pixel: only the scan here, the rays are placed in parallel
    // by k_rt_scatter and k_rt_sortcells
    rt_place(P, cs, c, sh_counts, s_chunk, active, P.Np != 1);
}

// parallel placement for one ray per pixel: each mapped ray takes a slot of
// its cell's segment by an atomic cursor (in no particular order) ...
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rt_scatter(const Prob<T>* __restrict__ probs,
                                                         const int* __restrict__ cand_prob,
                                                         const double* __restrict__ lens, int cand0, int chunk,
                                                         CandScratch<T> cs, int* __restrict__ cursor,
                                                         long long cursor_stride) {
    const int c = cand0 + blockIdx.y;
    const Prob<T>& P = probs[cand_prob[c]];
    if (P.Np != 1 || make_lens<double>(lens + 7LL * c).bad) return;
    const Entry<double>* Et = cs.Etmp + (long long)c * cs.sE;
    Entry<double>* E64 = cs.E64 + (long long)c * cs.sE;
    const int* cst = cs.cst + (long long)c * cs.sCst;
    int* cur = cursor + (long long)c * cursor_stride;
    int* inv = cs.inv + (long long)c * cs.sInv;
    const int r1 = min((int)(blockIdx.x + 1) * chunk, P.nrays);
    for (int r = blockIdx.x * chunk + threadIdx.x; r < r1; r += blockDim.x) {
        const Entry<double> e = Et[r];
        if (e.base >= 0) {
            const int iy0 = e.base / P.sx, ix0 = e.base - iy0 * P.sx;
            const int cell = iy0 * P.ncx + ix0;
            E64[cst[cell] + atomicAdd(&cur[cell], 1)] = e;
        } else {
            inv[r] = -1;
        }
    }
}

// ... then each cell's segment is sorted by ray index (the pixel's padded
// position is increasing in it), which is the stable order of the one-warp
// placement; the FP32 copy and the ray -> position index follow
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rt_sortcells(const Prob<T>* __restrict__ probs,
                                                           const int* __restrict__ cand_prob,
                                                           const double* __restrict__ lens, int cand0,
                                                           CandScratch<T> cs) {
    const int c = cand0 + blockIdx.y;
    const Prob<T>& P = probs[cand_prob[c]];
    if (P.Np != 1 || make_lens<double>(lens + 7LL * c).bad) return;
    Entry<double>* E64 = cs.E64 + (long long)c * cs.sE;
    Entry<T>* E = cs.E + (long long)c * cs.sE;
    const int* cst = cs.cst + (long long)c * cs.sCst;
    int* inv = cs.inv + (long long)c * cs.sInv;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= P.ncells) return;
    const int k0 = cst[cell], k1 = cst[cell + 1];
    for (int i = k0 + 1; i < k1; ++i) {  // insertion sort (cells hold few rays)
        const Entry<double> key = E64[i];
        int j = i - 1;
        while (j >= k0 && E64[j].ppos > key.ppos) {
            E64[j + 1] = E64[j];
            --j;
        }
        E64[j + 1] = key;
    }
    for (int i = k0; i < k1; ++i) {
        const Entry<double> e = E64[i];
        if ((void*)E != (void*)E64) {
            Entry<T> et;
            et.ppos = e.ppos;
            et.base = e.base;
            et.u = (T)e.u;
            et.v = (T)e.v;
            E[i] = et;
        }
        const int y = e.ppos / P.Wp - P.hk, x = e.ppos - (e.ppos / P.Wp) * P.Wp - P.xoff;
        inv[y * P.nx + x] = i;
    }
}

// ---------------------------------------------------------------------------
// Padded image layout.  Image pixel (x, y) lives at
//     pp(x, y) = (y + hk) * Wp + x + xoff,   xoff = hk rounded up to VW,
// so every 4-pixel tile row starts on a 16-byte boundary (conflict-free
// vector access) and a K x K window never leaves the zero-filled frame.
// Convolution of one TILE x TILE output tile at tile origin (X, Y):
//   out[r][c] = sum_{a,b} taps[a][b] * Pb[(Y + r + a) * Wp + X + c + b + sh]
// with Pb = buffer + 0, sh = xoff - hk.  taps = flipped PSF gives B,
// taps = PSF gives B^T (the blur operator of Section 2.2).
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr int vec_width() {
    return 16 / (int)sizeof(T);
}
template <typename T>
__host__ __device__ constexpr int xoff_of(int hk) {
    return (hk + vec_width<T>() - 1) / vec_width<T>() * vec_width<T>();
}

template <typename T, int K, bool SH>
__device__ __forceinline__ void conv_tile(const T* __restrict__ Pb, int Wp, const T* __restrict__ taps,
                                          T (&acc)[TILE][TILE]) {
    constexpr int VW = vec_width<T>();
    constexpr int HK = (K - 1) / 2;
    constexpr int SHF = xoff_of<T>(HK) - HK;
    constexpr int W = TILE + K - 1 + SHF;
    constexpr int NVW = (W + VW - 1) / VW * VW;
    constexpr int KP = (K + 3) & ~3;
    constexpr bool TAPREG = (K <= 9);
    const unsigned tap_a = smem_addr(taps);
    const unsigned src_a = SH ? smem_addr(Pb) : 0u;
    if constexpr (!TAPREG) {
        // larger PSFs: loop over pairs of tap rows; the pair's 2K taps are
        // loaded once, and window rows a..a+4 each once, serving tap row a
        // (output rows 0..3) and tap row a+1 (output rows 0..3 from window
        // rows a+1..a+4)
#pragma unroll
        for (int r = 0; r < TILE; ++r)
#pragma unroll
            for (int c = 0; c < TILE; ++c) acc[r][c] = 0;
#pragma unroll 1
        for (int a = 0; a + 1 < K; a += 2) {
            T t0[K], t1[K];
#pragma unroll
            for (int b = 0; b < K; ++b) {
                t0[b] = lds_one(tap_a + (unsigned)((a * KP + b) * sizeof(T)), T(0));
                t1[b] = lds_one(tap_a + (unsigned)(((a + 1) * KP + b) * sizeof(T)), T(0));
            }
#pragma unroll
            for (int rr = 0; rr <= TILE; ++rr) {
                T in[NVW];
#pragma unroll
                for (int v = 0; v < NVW; v += VW) {
                    if (SH)
                        lds_vec(src_a + (unsigned)(((a + rr) * Wp + v) * sizeof(T)), in + v);
                    else
                        vload(Pb + (a + rr) * Wp + v, in + v);
                }
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    if (rr < TILE) {
#pragma unroll
                        for (int c = 0; c < TILE; ++c) acc[rr][c] = fma(t0[b], in[SHF + b + c], acc[rr][c]);
                    }
                    if (rr >= 1) {
#pragma unroll
                        for (int c = 0; c < TILE; ++c) acc[rr - 1][c] = fma(t1[b], in[SHF + b + c], acc[rr - 1][c]);
                    }
                }
            }
        }
        if constexpr (K % 2 == 1) {  // the last tap row alone
            constexpr int a = K - 1;
            T t0[K];
#pragma unroll
            for (int b = 0; b < K; ++b) t0[b] = lds_one(tap_a + (unsigned)((a * KP + b) * sizeof(T)), T(0));
#pragma unroll
            for (int rr = 0; rr < TILE; ++rr) {
                T in[NVW];
#pragma unroll
                for (int v = 0; v < NVW; v += VW) {
                    if (SH)
                        lds_vec(src_a + (unsigned)(((a + rr) * Wp + v) * sizeof(T)), in + v);
                    else
                        vload(Pb + (a + rr) * Wp + v, in + v);
                }
#pragma unroll
                for (int b = 0; b < K; ++b)
#pragma unroll
                    for (int c = 0; c < TILE; ++c) acc[rr][c] = fma(t0[b], in[SHF + b + c], acc[rr][c]);
            }
        }
        return;
    }
    T tw[TAPREG ? K : 1][TAPREG ? K : 1];
    if constexpr (TAPREG) {
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
            for (int b = 0; b < K; ++b) tw[a][b] = lds_one(tap_a + (unsigned)((a * KP + b) * sizeof(T)), T(0));
    }
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
        // b outer, r inner: consecutive updates of one accumulator are up to
        // 16 FMAs apart, which hides the FMA latency within one warp
#pragma unroll
        for (int b = 0; b < K; ++b) {
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int a = i - r;
                if (a >= 0 && a < K) {
                    T t;
                    if constexpr (TAPREG)
                        t = tw[a][b];
                    else
                        t = lds_one(tap_a + (unsigned)((a * KP + b) * sizeof(T)), T(0));
#pragma unroll
                    for (int c = 0; c < TILE; ++c) acc[r][c] = fma(t, in[c + b + SHF], acc[r][c]);
                }
            }
        }
    }
}

// runtime-K tile (any type, any address space); also the FP64 path of the
// mixed-precision refinement
template <typename S, typename U>
__device__ __forceinline__ void conv_tile_rt(const S* __restrict__ Pb, int Wp, const U* __restrict__ taps, int K,
                                             int KP, int sh, S (&acc)[TILE][TILE]) {
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int c = 0; c < TILE; ++c) acc[r][c] = 0;
    for (int a = 0; a < K; ++a) {
        for (int b = 0; b < K; ++b) {
            const S t = (S)taps[a * KP + b];
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const S* row = Pb + (r + a) * Wp + b + sh;
#pragma unroll
                for (int c = 0; c < TILE; ++c) acc[r][c] = fma(t, row[c], acc[r][c]);
            }
        }
    }
}

// (Geo: reg.cuh)

template <typename T>
__device__ __forceinline__ Geo<T> geo_of(const Prob<T>& P, int nent) {
    Geo<T> g;
    g.nx = P.nx;
    g.ny = P.ny;
    g.sx = P.sx;
    g.sy = P.sy;
    g.ns = P.ns;
    g.nreg = P.nreg;
    g.K = P.K;
    g.hk = P.hk;
    g.kp = P.kp;
    g.xoff = P.xoff;
    g.sh = P.xoff - P.hk;
    g.Np = P.Np;
    g.ncx = P.ncx;
    g.ncells = P.ncells;
    g.Wp = P.Wp;
    g.plen = P.plen;
    g.tiles_x = P.tiles_x;
    g.ntiles = P.ntiles;
    g.reg = P.reg;
    g.nent = nent;
    g.interp = P.interp;
    g.invNp = P.invNp;
    return g;
}

// work buffers of one item
// FFT plans of one item: inner solves (T) and refinement (FP64)
template <typename T>
struct FftPair {
    FftPlan<T> t;
    FftPlan<double> d;
};
static_assert(sizeof(FftPair<float>) <= 128 && sizeof(FftPair<double>) <= 128, "FFT plans exceed their 128 bytes");

template <typename T>
struct Work {
    T* taps;          // [2][K][kp]: flipped PSF (B), PSF (B^T)
    double* taps64;   // same taps in double (refinement path)
    T* swp;           // [plen] sqrt(W) = m / sigma
    const T* dpad;    // [plen] observed image (padded, global)
    T* rimg;          // [plen] inner residual (image part)
    T* qimg;          // [plen] sqrt(W) B L p, then u = B^T sqrt(W) r
    T* P1;            // [plen] L p (zero frame)
    T* P2;            // [plen] sqrt(W) r (zero frame)
    const Entry<T>* E;
    const Entry<double>* E64;  // FP64-weight copy (global) for the refinement
    const int* inv;   // only for sub-pixel problems
    const int* cst;
    T* x;             // [ns] inner iterate (correction)
    T* p;
    T* s;
    T* rreg;          // [nreg]
    T* qreg;
    T* minv;          // [ns] Jacobi preconditioner of the inner solves
    double* x64;      // [ns] solution accumulator (refinement)
    double* xb;       // [ns] the refinement iterate with the smallest true residual so far
    double* h64;      // [nreg] H x64
    double* Pa;       // [plen] L x64
    double* Pb;       // [plen] sqrt(W) r64
    double* Pc;       // [plen] B^T sqrt(W) r64
    const FftPair<T>* fft = nullptr;  // shared: the FFT plans when the problem convolves by FFT, else null
};

// one ray's bicubic sample of v (without the 1/N_p)
template <typename T, typename ET, typename V>
__device__ __forceinline__ V bicubic_sample(const Geo<T>& g, const Entry<ET>& en, const V* __restrict__ v) {
    const int iy0 = en.base / g.sx, ix0 = en.base - iy0 * g.sx;
    V acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = iy0 - 1 + j;
        if (y < 0 || y >= g.sy) continue;
        V row = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = ix0 - 1 + i;
            if (x >= 0 && x < g.sx) row += keys_weight(i, (V)en.u) * v[y * g.sx + x];
        }
        acc += keys_weight(j, (V)en.v) * row;
    }
    return acc;
}

// L v for bicubic rays (out of line, like the two below: kernels that also
// run bilinear problems keep their register allocation)
template <typename T, typename ET, typename V, typename D>
__device__ __noinline__ void bicubic_L(const Geo<T>& g, const Entry<ET>* __restrict__ Ent, const int* __restrict__ inv,
                                       const V* __restrict__ v, D* __restrict__ dst) {
    if (g.Np == 1) {
        for (int k = threadIdx.x; k < g.nent; k += blockDim.x) {
            const Entry<ET> en = Ent[k];
            dst[en.ppos] = (D)bicubic_sample(g, en, v);
        }
        return;
    }
    const int npix = g.nx * g.ny;
    for (int j = threadIdx.x; j < npix; j += blockDim.x) {
        V val = 0;
        int pp = -1;
        for (int a = 0; a < g.Np; ++a) {
            const int e = inv[j * g.Np + a];
            if (e >= 0) {
                const Entry<ET> en = Ent[e];
                val += bicubic_sample(g, en, v);
                pp = en.ppos;
            }
        }
        if (pp >= 0) dst[pp] = (D)(val * (V)g.invNp);
    }
}

// (L^T U)_i for bicubic rays: the 4 x 4 cells whose rays reach (ia, ib), in
// a fixed order
template <typename T, typename ET, typename V>
__device__ __noinline__ V bicubic_LT_at(const Geo<T>& g, const Entry<ET>* __restrict__ Ent,
                                        const int* __restrict__ cst, const V* __restrict__ U, int ia, int ib) {
    V acc = 0;
    for (int j = 0; j < 4; ++j) {
        const int iy0 = ib + 1 - j;
        if (iy0 < 0 || iy0 > g.sy - 2) continue;
        for (int i = 0; i < 4; ++i) {
            const int ix0 = ia + 1 - i;
            if (ix0 < 0 || ix0 > g.sx - 2) continue;
            const int cell = iy0 * g.ncx + ix0;
            const int k1 = cst[cell + 1];
            for (int k = cst[cell]; k < k1; ++k) {
                const Entry<ET> en = Ent[k];
                acc += keys_weight(i, (V)en.u) * keys_weight(j, (V)en.v) * U[en.ppos];
            }
        }
    }
    return acc * (V)g.invNp;
}

// dst <- L v (Section 2.2: interpolation of the back-traced rays, averaged
// over sub-pixels; bilinear, or nearest neighbour through snapped offsets,
// or bicubic).  Only mapped pixels are written; the rest of dst must hold
// zeros.
template <typename T, typename ET, typename V, typename D>
__device__ __forceinline__ void apply_L(const Geo<T>& g, const Entry<ET>* __restrict__ Ent, const int* __restrict__ inv,
                                        const V* __restrict__ v, D* __restrict__ dst) {
    if (g.interp == 2) {
        bicubic_L(g, Ent, inv, v, dst);
        return;
    }
    if (g.Np == 1) {
        for (int k = threadIdx.x; k < g.nent; k += blockDim.x) {
            const Entry<ET> en = Ent[k];
            const V u = (V)en.u, vv = (V)en.v;
            const V* s0 = v + en.base;
            dst[en.ppos] = (D)(((V)1 - vv) * (((V)1 - u) * s0[0] + u * s0[1]) +
                               vv * (((V)1 - u) * s0[g.sx] + u * s0[g.sx + 1]));
        }
        return;
    }
    const int npix = g.nx * g.ny;
    for (int j = threadIdx.x; j < npix; j += blockDim.x) {
        V val = 0;
        int pp = -1;
        for (int a = 0; a < g.Np; ++a) {
            const int e = inv[j * g.Np + a];
            if (e >= 0) {
                const Entry<ET> en = Ent[e];
                const V u = (V)en.u, vv = (V)en.v;
                const V* s0 = v + en.base;
                val += ((V)1 - vv) * (((V)1 - u) * s0[0] + u * s0[1]) + vv * (((V)1 - u) * s0[g.sx] + u * s0[g.sx + 1]);
                pp = en.ppos;
            }
        }
        if (pp >= 0) dst[pp] = (D)(val * (V)g.invNp);
    }
}

// (L^T U)_i: gather over the rays of the (up to) four cells having source
// pixel (ia, ib) as a corner, in sorted (deterministic) order
// (BICUBIC = false: a caller that never sees bicubic rays skips the branch)
template <typename T, typename ET, typename V, bool BICUBIC = true>
__device__ __forceinline__ V apply_LT_at(const Geo<T>& g, const Entry<ET>* __restrict__ Ent,
                                         const int* __restrict__ cst, const V* __restrict__ U, int ia, int ib) {
    if (BICUBIC && g.interp == 2) return bicubic_LT_at(g, Ent, cst, U, ia, ib);
    V acc = 0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int iy0 = ib - dy;
        if (iy0 < 0 || iy0 > g.sy - 2) continue;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int ix0 = ia - dx;
            if (ix0 < 0 || ix0 > g.sx - 2) continue;
            const int cell = iy0 * g.ncx + ix0;
            const int k1 = cst[cell + 1];
            for (int k = cst[cell]; k < k1; ++k) {
                const Entry<ET> en = Ent[k];
                const V wu = dx ? (V)en.u : (V)1 - (V)en.u;
                const V wv = dy ? (V)en.v : (V)1 - (V)en.v;
                acc += wu * wv * U[en.ppos];
            }
        }
    }
    return acc * (V)g.invNp;
}

// (apply_H_row, apply_HT_at: reg.cuh)

// lwl_diag_at for bicubic rays
template <typename T>
__device__ __noinline__ T bicubic_diag_at(const Geo<T>& g, const Entry<T>* __restrict__ Ent,
                                          const int* __restrict__ cst, const double* __restrict__ omega, int ia,
                                          int ib) {
    T acc = 0;
    for (int j = 0; j < 4; ++j) {
        const int iy0 = ib + 1 - j;
        if (iy0 < 0 || iy0 > g.sy - 2) continue;
        for (int i = 0; i < 4; ++i) {
            const int ix0 = ia + 1 - i;
            if (ix0 < 0 || ix0 > g.sx - 2) continue;
            const int cell = iy0 * g.ncx + ix0;
            const int k1 = cst[cell + 1];
            for (int k = cst[cell]; k < k1; ++k) {
                const Entry<T> en = Ent[k];
                const T wt = keys_weight(i, en.u) * keys_weight(j, en.v) * g.invNp;
                acc += wt * wt * (T)omega[en.ppos];
            }
        }
    }
    return acc;
}

// Approximate diagonal of the inner normal operator L^T B^T W B L at source
// pixel (ia, ib): sum over the rays of its cells of (bilinear weight / N_p)^2
// times omega at the ray's pixel, omega_p = diag(B^T W B)_p = sum_k psf_k^2
// W_{p+k-c} (the weight the PSF spreads pixel p's light over).  It drops the
// off-diagonal terms of B^T W B and the cross terms between rays; it is exact
// for a delta PSF, and near a mask edge it keeps the light the PSF carries
// into unmasked pixels.
template <typename T>
__device__ __forceinline__ T lwl_diag_at(const Geo<T>& g, const Entry<T>* __restrict__ Ent, const int* __restrict__ cst,
                                         const double* __restrict__ omega, int ia, int ib) {
    if (g.interp == 2) return bicubic_diag_at(g, Ent, cst, omega, ia, ib);
    T acc = 0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int iy0 = ib - dy;
        if (iy0 < 0 || iy0 > g.sy - 2) continue;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int ix0 = ia - dx;
            if (ix0 < 0 || ix0 > g.sx - 2) continue;
            const int cell = iy0 * g.ncx + ix0;
            const int k1 = cst[cell + 1];
            for (int k = cst[cell]; k < k1; ++k) {
                const Entry<T> en = Ent[k];
                const T wu = dx ? en.u : (T)1 - en.u;
                const T wv = dy ? en.v : (T)1 - en.v;
                const T wt = wu * wv * g.invNp;
                acc += wt * wt * (T)omega[en.ppos];
            }
        }
    }
    return acc;
}

// (hth_diag_at: reg.cuh)

// 4-wide vector helpers for one tile row (float: one 16-byte access;
// double: two)
template <typename T>
struct V4 {
    T v[4];
};
template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
    V4<T> o;
    vload(p, o.v);
    if (sizeof(T) == 8) vload(p + 2, o.v + 2);
    return o;
}
__device__ __forceinline__ void st4(float* p, const V4<float>& o) {
    *reinterpret_cast<float4*>(p) = make_float4(o.v[0], o.v[1], o.v[2], o.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& o) {
    *reinterpret_cast<double2*>(p) = make_double2(o.v[0], o.v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(o.v[2], o.v[3]);
}

enum : int { CONV_Q = 0, CONV_RAW = 1 };

// One convolution over all owned tiles (one non-inlined copy of the
// unrolled tile code per kernel):
//   CONV_Q   : dst = sqrt(W) * conv, returns sum dst^2
//   CONV_RAW : dst = conv
template <typename T, int K, bool SH>
__device__ __noinline__ T conv_pass(const T* __restrict__ src, const T* __restrict__ taps,
                                         const T* __restrict__ swp, T* __restrict__ dst, Geo<T> g, int mode) {
    T ss = 0;
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
        const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
        T acc[TILE][TILE];
        const T* base = src + (ty * TILE) * g.Wp + tx * TILE;
        if constexpr (K > 0)
            conv_tile<T, K, SH>(base, g.Wp, taps, acc);
        else
            conv_tile_rt<T, T>(base, g.Wp, taps, g.K, g.kp, g.sh, acc);
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + g.xoff;
            V4<T> o;
            if (mode == CONV_Q) {
                const V4<T> sw = ld4(swp + pp);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    o.v[c] = sw.v[c] * acc[r][c];
                    ss = fma(o.v[c], o.v[c], ss);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) o.v[c] = acc[r][c];
            }
            st4(dst + pp, o);
        }
    }
    return ss;
}

// FP64 convolution pass of the refinement:
//   mode 0: res = sqrt(W)(d - conv(Pa)); rimg = (T)res; Pb = sqrt(W) res; returns sum res^2
//   mode 1: Pc = conv(Pb)
template <typename T>
__device__ __noinline__ double conv64_pass(const Work<T> w, Geo<T> g, int mode) {
    double ss = 0;
    if (w.fft) {  // the same passes through the FFT convolution
        const double* src = mode == 0 ? w.Pa : w.Pb;
        auto load = [&](int y, int n) -> double { return n < g.nx ? src[(y + g.hk) * g.Wp + n + g.xoff] : 0.0; };
        auto store = [&](int y, int n, double v) {
            const int pp = (y + g.hk) * g.Wp + n + g.xoff;
            if (mode == 0) {
                const double sw = (double)w.swp[pp];
                const double res = sw * ((double)w.dpad[pp] - v);
                w.rimg[pp] = (T)res;
                w.Pb[pp] = sw * res;
                ss += res * res;
            } else {
                w.Pc[pp] = v;
            }
        };
        fft_convolve<double>(w.fft->d, load, g.ny, store, g.ny, g.nx, mode != 0);
        return ss;
    }
    const double* src = mode == 0 ? w.Pa : w.Pb;
    const double* taps = w.taps64 + (mode == 0 ? 0 : g.K * g.kp);
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
        const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
        double acc[TILE][TILE];
        conv_tile_rt<double, double>(src + (ty * TILE) * g.Wp + tx * TILE, g.Wp, taps, g.K, g.kp, g.sh, acc);
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
            const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + g.xoff;
#pragma unroll
            for (int c = 0; c < TILE; ++c) {
                if (mode == 0) {
                    const double sw = (double)w.swp[pp + c];
                    const double res = sw * ((double)w.dpad[pp + c] - acc[r][c]);
                    w.rimg[pp + c] = (T)res;
                    w.Pb[pp + c] = sw * res;
                    ss += res * res;
                } else {
                    w.Pc[pp + c] = acc[r][c];
                }
            }
        }
    }
    return ss;
}

// conv_pass through the FFT convolution (B for CONV_Q, B^T for CONV_RAW);
// writes image pixels only (the frame keeps the zeros set at item start)
template <typename T>
__device__ __noinline__ T conv_pass_fft(const FftPlan<T>* f, const T* __restrict__ src, const T* __restrict__ swp,
                                        T* __restrict__ dst, Geo<T> g, int mode) {
    T ss = 0;
    auto load = [&](int y, int n) -> T { return n < g.nx ? src[(y + g.hk) * g.Wp + n + g.xoff] : (T)0; };
    auto store = [&](int y, int n, T v) {
        const int pp = (y + g.hk) * g.Wp + n + g.xoff;
        if (mode == CONV_Q) {
            const T o = swp[pp] * v;
            dst[pp] = o;
            ss = fma(o, o, ss);
        } else {
            dst[pp] = v;
        }
    };
    fft_convolve<T>(*f, load, g.ny, store, g.ny, g.nx, mode != CONV_Q);
    return ss;
}

// FP64 residual of the current solution x64 (the refinement step):
//   r = [sqrt(W)(d - B L x64); -sqrt(lam) H x64],  s = A~^T r = rhs - A x64.
// Writes the inner-solve start: rimg, rreg, s (type T).  Returns chi2 =
// ||r_img||^2 and sets reg2 = ||H x64||^2 and g64 = ||s||^2.
// The refinement's FP64 convolution passes in FP32 contexts as double-float
// sums on the FP32 pipe (dfloat.cuh; the taps are FP32 numbers): about 11
// FP32 operations per tap instead of one FP64 FMA at 1/64 of the FP32
// rate, ~2^-44 relative.  hi and lo are staged in the P1/P2 image buffers,
// which hold zeros again on return.  KT > 0: compiled tap count.
template <int KT>
__device__ __noinline__ double conv64_df_gen(const double* __restrict__ src, float* __restrict__ hi,
                                             float* __restrict__ lo, const float* __restrict__ taps,
                                             const float* __restrict__ swp, const float* __restrict__ dpad,
                                             float* __restrict__ rimg, double* __restrict__ Pb,
                                             double* __restrict__ Pc, const Geo<float> g, int mode) {
    for (int i = threadIdx.x; i < g.plen; i += blockDim.x) df_split(src[i], hi[i], lo[i]);
    __syncthreads();
    const int K = KT > 0 ? KT : g.K, kp = g.kp;
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
                const float* trow = taps + a * kp;
                if constexpr (KT > 0) {
                    float xh[KT + TILE - 1], xl[KT + TILE - 1];
#pragma unroll
                    for (int j = 0; j < KT + TILE - 1; ++j) {
                        xh[j] = hrow[j];
                        xl[j] = lrow[j];
                    }
#pragma unroll
                    for (int b = 0; b < KT; ++b) {
                        const float tt = trow[b];
#pragma unroll
                        for (int q = 0; q < TILE; ++q) df_madd(s[q], c[q], tt, xh[b + q], xl[b + q]);
                    }
                } else {
#pragma unroll 1
                    for (int b = 0; b < K; ++b) {
                        const float tt = trow[b];
#pragma unroll
                        for (int q = 0; q < TILE; ++q) df_madd(s[q], c[q], tt, hrow[b + q], lrow[b + q]);
                    }
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

// the general kernel's refinement passes: double-float for direct
// convolution in FP32 contexts, conv64_pass otherwise (FP64 contexts, FFT)
template <typename T, int KT>
struct Conv64Gen {
    __device__ double operator()(const Work<T>& w, const Geo<T>& g, int mode) const {
        if constexpr (sizeof(T) == 4) {
            if (!w.fft)
                return conv64_df_gen<KT>(mode == 0 ? w.Pa : w.Pb, w.P1, w.P2, w.taps + (mode == 0 ? 0 : g.K * g.kp),
                                         w.swp, w.dpad, w.rimg, w.Pb, w.Pc, g, mode);
        }
        return conv64_pass<T>(w, g, mode);
    }
};

// conv: the refinement's two convolution passes (mode 0: the image residual
// from L x64, mode 1: B^T of the weighted residual) as each kernel forms them
template <typename T, class Conv>
__device__ __forceinline__ double residual64(const Work<T>& w, const Geo<T>& g, double lam, double* red,
                                             int& which, double& reg2, double& g64, const Conv& conv) {
    apply_L<T, double, double, double>(g, w.E64, w.inv, w.x64, w.Pa);
    const double sl = sqrt(lam);
    double rg = 0;
    for (int i = threadIdx.x; i < g.nreg; i += blockDim.x) {
        const double h = apply_H_row<T, double>(g, w.x64, i);
        w.h64[i] = h;
        w.rreg[i] = (T)(-sl * h);
        rg += h * h;
    }
    __syncthreads();
    const double chi2 = block_sum(conv(w, g, 0), red, which);
    which ^= 1;
    conv(w, g, 1);
    __syncthreads();
    double ss = 0;
    for (int i = threadIdx.x; i < g.ns; i += blockDim.x) {
        const int ib = i / g.sx, ia = i - ib * g.sx;
        const double v = apply_LT_at<T, double, double>(g, w.E64, w.cst, w.Pc, ia, ib) -
                         lam * apply_HT_at<T, double>(g, w.h64, i, ia, ib);
        w.s[i] = (T)v;
        ss += v * v;
    }
    g64 = block_sum(ss, red, which);
    which ^= 1;
    reg2 = block_sum(rg, red, which);
    which ^= 1;
    return chi2;
}

// ---------------------------------------------------------------------------
// k_cgls: persistent CTAs, one (candidate, lambda) item at a time.
// Each item solves min ||sqrt(W)(B L s - d)||^2 + lam ||H s||^2 by
// iterative refinement: an FP64 residual r = b~ - A~ x (Eq. chi2 and the
// regulariser of Eq. TKReg, with x the FP64 solution), then CGLS in type T
// on A~ dx = r (inner solve, Section 2.2 / 2.4 CGLS started from a blank
// correction), x += dx; until ||A~^T r|| <= tol ||A~^T b~||.  In T = double
// contexts the first inner solve normally reaches the tolerance.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t align_up(size_t v, size_t a) {
    return (v + a - 1) / a * a;
}

// Placement of the work buffers of the general CGLS kernel:
//   PLACE_SMEM   everything in shared memory (small images)
//   PLACE_GLOBAL everything in a per-CTA global slab (L2-resident)
//   PLACE_MID    the two convolution inputs and the source vectors in
//                shared memory, the rest in the slab (mid-size images)
// In FP32 contexts each inner solve of the refinement aims for max(eta,
// FINAL_MARGIN tol / current residual): the last one stops where the FP64
// residual is expected at FINAL_MARGIN of the tolerance.  0.8 leaves room
// for the difference between the FP32 recursion's residual and the FP64 one
// (measured: every item of the benchmark batch still met the tolerance in
// that pass, largest residual 0.998 tol) and is 5% faster than 0.3.  FP64
// contexts, whose single inner solve normally reaches the tolerance, keep
// the margin FINAL_MARGIN64.  Every solve still aims for at least a
// reduction by MAX_TARGET: a residual just above the tolerance (a warm
// start) would otherwise ask for a reduction near 1, and two such steps in
// a row read as stagnation.
constexpr double FINAL_MARGIN = 0.8, FINAL_MARGIN64 = 0.3, MAX_TARGET = 0.5;

enum : int { PLACE_SMEM = 0, PLACE_GLOBAL = 1, PLACE_MID = 2 };
// kernel-table indices of the global-slab and split kernels compiled for two
// CTAs per SM (their buffers are laid out as PLACE_GLOBAL and PLACE_MID)
constexpr int PLACE_GLOBAL2 = 3, PLACE_MID2 = 4;
__host__ __device__ constexpr int layout_of(int place) {
    return place == PLACE_GLOBAL2 ? PLACE_GLOBAL : place == PLACE_MID2 ? PLACE_MID : place;
}
__host__ __device__ constexpr bool two_per_sm(int place) { return place == PLACE_GLOBAL2 || place == PLACE_MID2; }

template <typename T>
__host__ __device__ inline size_t smem_bytes(const Prob<T>& P, int place) {
    size_t o = 16 + 2 * 33 * sizeof(double) + 128;                 // item slot + reductions + CG scalars
    o += align_up<T>(sizeof(T) * 2 * P.K * P.kp, 16);              // taps
    o += align_up<T>(sizeof(double) * 2 * P.K * P.kp, 16);         // taps64
    if (place == PLACE_SMEM) {
        o += 5 * align_up<T>(sizeof(T) * P.plen, 16);                  // swp rimg qimg P1 P2
        o += align_up<T>(sizeof(Entry<T>) * (size_t)P.nrays, 16);      // E
        if (P.Np > 1) o += align_up<T>(sizeof(int) * (size_t)P.nrays, 16);  // inv
        o += align_up<T>(sizeof(int) * (size_t)(P.ncells + 1), 16);    // cst
    } else if (place == PLACE_MID) {
        o += 2 * align_up<T>(sizeof(T) * P.plen, 16);                  // P1 P2
    }
    if (place != PLACE_GLOBAL) {
        o += 4 * align_up<T>(sizeof(T) * P.ns, 16);                    // x p s minv
        o += 2 * align_up<T>(sizeof(T) * P.nreg, 16);                  // rreg qreg
    }
    if (P.fft_m) o += fft_smem_bytes(P.fft_m);                         // FFT twiddles and batch buffers
    return o;
}

// per-CTA global slab: [double part][T part], in bytes
template <typename T>
__host__ __device__ inline size_t slab_bytes(const Prob<T>& P, int place) {
    size_t o = sizeof(double) * (3 * align_up<T>(P.plen, 4) + 2 * align_up<T>(P.ns, 4) + align_up<T>(P.nreg, 4));
    if (place == PLACE_GLOBAL)
        o += sizeof(T) * (4 * align_up<T>(P.plen, 4) + 4 * align_up<T>(P.ns, 4) + 2 * align_up<T>(P.nreg, 4));
    if (place == PLACE_MID) o += sizeof(T) * 2 * align_up<T>(P.plen, 4);  // rimg qimg
    if (P.fft_m) o += 16 + sizeof(double2) * (size_t)((P.fft_m >> 1) + 1) * P.fft_m;  // FFT work spectra
    return align_up<T>(o, 256);
}

// A work item of the CGLS kernels is a chain of one candidate's lambdas,
// solved in order by one CTA: packed = (c * MAX_LAM + k_first) * MAX_LAM +
// k_last (a single lambda has k_first == k_last).  After the first lambda of
// a chain, each solve starts from the previous lambda's solution, which is
// still in the CTA's FP64 accumulator (unless that solve broke down).  Every
// thread holds the same state and takes the same steps.
struct ChainPos {
    int c = 0, k = 0, k_last = -1, step = 1;
    bool warm = false;     // the current lambda continues a chain
    bool prev_ok = false;  // the previous lambda's solution is usable
    __device__ bool next() {
        if (k_last < 0 || k == k_last) return false;
        k += step;
        warm = true;
        return true;
    }
    __device__ void start(int packed) {
        c = packed / (MAX_LAM * MAX_LAM);
        const int r = packed - c * (MAX_LAM * MAX_LAM);
        k = r / MAX_LAM;
        k_last = r - k * MAX_LAM;
        step = k_last >= k ? 1 : -1;
        warm = false;
        prev_ok = false;
    }
};

// MINB: resident CTAs per SM the register allocation is held to (2 caps
// it at 128 registers a thread, so that two latency-bound global-slab CTAs
// share an SM)
template <typename T, int K, int PLACE, int MINB = 1>
__global__ void __launch_bounds__(NTHREADS, MINB) k_cgls(CglsArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool BIG = PLACE == PLACE_GLOBAL;
    constexpr bool MID = PLACE == PLACE_MID;
    constexpr bool SH = !BIG;  // convolution inputs in shared memory
    const int tid = threadIdx.x, bs = blockDim.x;
    int last_c = -1;
    int which = 0;
    int* slot = reinterpret_cast<int*>(smem);
    double* red = reinterpret_cast<double*>(smem + 16);
    CgCtl* ctl = reinterpret_cast<CgCtl*>(smem + 16 + 2 * 33 * sizeof(double));
    ChainPos ch;

    while (true) {
        __syncthreads();
        if (!ch.next()) {
            if (tid == 0) slot[0] = atomicAdd(A.counter, 1);
            __syncthreads();
            const int it_idx = slot[0];
            if (it_idx >= A.n_items) break;
            ch.start(A.items[it_idx]);
        }
        const int c = ch.c, k = ch.k;
        const Prob<T>& P = A.probs[A.cand_prob[c]];
        const CandScratch<T>& cs = A.cs;
        const int nent = cs.nent[c];
        const Geo<T> g = geo_of(P, nent);

        // ---- carve buffers
        Work<T> w;
        unsigned char* fslab = nullptr;
        unsigned char* sp = smem + 16 + 2 * 33 * sizeof(double) + 128;
        w.taps = reinterpret_cast<T*>(sp);
        sp += align_up<T>(sizeof(T) * 2 * g.K * g.kp, 16);
        w.taps64 = reinterpret_cast<double*>(sp);
        sp += align_up<T>(sizeof(double) * 2 * g.K * g.kp, 16);
        const T* g_swp = cs.swp + (long long)c * cs.sPad;
        w.dpad = cs.dpad + (long long)c * cs.sPad;
        const Entry<T>* g_E = cs.E + (long long)c * cs.sE;
        w.E64 = cs.E64 + (long long)c * cs.sE;
        const int* g_inv = cs.inv + (long long)c * cs.sInv;
        const int* g_cst = cs.cst + (long long)c * cs.sCst;
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
        if constexpr (PLACE == PLACE_SMEM) {
            const size_t pl = align_up<T>(sizeof(T) * g.plen, 16);
            w.swp = reinterpret_cast<T*>(sp); sp += pl;
            w.rimg = reinterpret_cast<T*>(sp); sp += pl;
            w.qimg = reinterpret_cast<T*>(sp); sp += pl;
            w.P1 = reinterpret_cast<T*>(sp); sp += pl;
            w.P2 = reinterpret_cast<T*>(sp); sp += pl;
            Entry<T>* sE = reinterpret_cast<Entry<T>*>(sp);
            sp += align_up<T>(sizeof(Entry<T>) * (size_t)P.nrays, 16);
            int* sInv = nullptr;
            if (g.Np > 1) {
                sInv = reinterpret_cast<int*>(sp);
                sp += align_up<T>(sizeof(int) * (size_t)P.nrays, 16);
            }
            int* sCst = reinterpret_cast<int*>(sp);
            sp += align_up<T>(sizeof(int) * (size_t)(P.ncells + 1), 16);
            const size_t ps = align_up<T>(sizeof(T) * g.ns, 16);
            const size_t pr = align_up<T>(sizeof(T) * g.nreg, 16);
            w.x = reinterpret_cast<T*>(sp); sp += ps;
            w.p = reinterpret_cast<T*>(sp); sp += ps;
            w.s = reinterpret_cast<T*>(sp); sp += ps;
            w.minv = reinterpret_cast<T*>(sp); sp += ps;
            w.rreg = reinterpret_cast<T*>(sp); sp += pr;
            w.qreg = reinterpret_cast<T*>(sp); sp += pr;
            w.E = sE;
            w.inv = sInv;
            w.cst = sCst;
            if (c != last_c) {
                // stage the candidate's lens operator and weights in shared memory
                for (int i = tid; i < nent; i += bs) sE[i] = g_E[i];
                if (g.Np > 1)
                    for (int i = tid; i < P.nrays; i += bs) sInv[i] = g_inv[i];
                for (int i = tid; i <= P.ncells; i += bs) sCst[i] = g_cst[i];
                for (int i = tid; i < g.plen; i += bs) w.swp[i] = g_swp[i];
            }
        } else if constexpr (MID) {
            const size_t pl = align_up<T>(sizeof(T) * g.plen, 16);
            w.P1 = reinterpret_cast<T*>(sp); sp += pl;
            w.P2 = reinterpret_cast<T*>(sp); sp += pl;
            const size_t ps = align_up<T>(sizeof(T) * g.ns, 16);
            const size_t pr = align_up<T>(sizeof(T) * g.nreg, 16);
            w.x = reinterpret_cast<T*>(sp); sp += ps;
            w.p = reinterpret_cast<T*>(sp); sp += ps;
            w.s = reinterpret_cast<T*>(sp); sp += ps;
            w.minv = reinterpret_cast<T*>(sp); sp += ps;
            w.rreg = reinterpret_cast<T*>(sp); sp += pr;
            w.qreg = reinterpret_cast<T*>(sp); sp += pr;
            T* ts = reinterpret_cast<T*>(slab);
            const size_t pg = align_up<T>(g.plen, 4);
            w.rimg = ts; ts += pg;
            w.qimg = ts; ts += pg;
            w.swp = const_cast<T*>(g_swp);
            w.E = g_E;
            w.inv = g_inv;
            w.cst = g_cst;
        } else {
            T* ts = reinterpret_cast<T*>(slab);
            const size_t pl = align_up<T>(g.plen, 4);
            w.rimg = ts; ts += pl;
            w.qimg = ts; ts += pl;
            w.P1 = ts; ts += pl;
            w.P2 = ts; ts += pl;
            w.x = ts; ts += align_up<T>(g.ns, 4);
            w.p = ts; ts += align_up<T>(g.ns, 4);
            w.s = ts; ts += align_up<T>(g.ns, 4);
            w.minv = ts; ts += align_up<T>(g.ns, 4);
            w.rreg = ts; ts += align_up<T>(g.nreg, 4);
            w.qreg = ts; ts += align_up<T>(g.nreg, 4);
            w.swp = const_cast<T*>(g_swp);
            w.E = g_E;
            w.inv = g_inv;
            w.cst = g_cst;
            fslab = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(ts) + 15) & ~uintptr_t(15));
        }
        // FFT convolution (runtime-K global-memory kernel only): twiddles and
        // batch buffers after the taps in shared memory, the work spectra at
        // the end of the slab, the problem's PSF spectra from the arguments
        w.fft = nullptr;
        if constexpr (K == 0 && BIG) {
            if (P.fft_m) {
                const int M = P.fft_m, pi = A.cand_prob[c];
                unsigned char* fs = sp;
                FftPair<T>* pp = reinterpret_cast<FftPair<T>*>(fs);
                fs += 128;
                float2* tw32 = reinterpret_cast<float2*>(fs);
                fs += align_up<T>(sizeof(float2) * (M - 1), 16);
                double2* tw64 = reinterpret_cast<double2*>(fs);
                fs += align_up<T>(sizeof(double2) * (M - 1), 16);
                using CT = typename CxOf<T>::type;
                if (tid == 0) {  // read after the barrier that ends the item set-up
                    FftPlan<T> a;
                    FftPlan<double> b;
                    a.M = b.M = M;
                    a.logM = b.logM = P.fft_log;
                    a.nb = fft_batch_count<CT>(M);
                    b.nb = fft_batch_count<double2>(M);
                    a.b0 = reinterpret_cast<CT*>(fs);
                    a.b1 = a.b0 + a.nb * (M + 1);
                    b.b0 = reinterpret_cast<double2*>(fs);
                    b.b1 = b.b0 + b.nb * (M + 1);
                    a.F = reinterpret_cast<CT*>(fslab);
                    b.F = reinterpret_cast<double2*>(fslab);
                    b.S = A.spec64 + (long long)pi * A.spec_stride;
                    b.tw = tw64;
                    if constexpr (sizeof(T) == 4) {
                        a.S = A.spec32 + (long long)pi * A.spec_stride;
                        a.tw = tw32;
                    } else {
                        a.S = A.spec64 + (long long)pi * A.spec_stride;
                        a.tw = tw64;
                    }
                    pp->t = a;
                    pp->d = b;
                }
                w.fft = pp;
                if (c != last_c) {
                    fft_twiddles<float>(tw32, M);
                    fft_twiddles<double>(tw64, M);
                }
            }
        }
        if (c != last_c) {
            // taps: [0] flipped PSF for B, [1] PSF for B^T; rows padded to kp
            for (int i = tid; i < 2 * g.K * g.kp; i += bs) {
                const int h = i / (g.K * g.kp), rem = i - h * g.K * g.kp;
                const int a = rem / g.kp, b = rem - a * g.kp;
                T v = 0;
                if (b < g.K) v = h == 0 ? P.psf[(g.K - 1 - a) * g.K + (g.K - 1 - b)] : P.psf[a * g.K + b];
                w.taps[i] = v;
                w.taps64[i] = (double)v;
            }
        }
        last_c = c;
        for (int i = tid; i < g.plen; i += bs) {
            w.P1[i] = 0;
            w.P2[i] = 0;
            w.Pa[i] = 0;
            w.Pb[i] = 0;
            if (w.fft) {  // the FFT passes write image pixels only: the frame stays zero
                w.rimg[i] = 0;
                w.qimg[i] = 0;
            }
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
            ch.prev_ok = false;
            continue;
        }

        const double lam = A.lambdas[(long long)c * A.max_lam + k];
        const T sl = (T)sqrt(lam);
        const int maxit = A.maxit > 0 ? A.maxit : 25 * g.ns;

        // ---- ||rhs|| = ||L^T B^T W d|| in FP64 (Pb = sqrt(W) sqrt(W) d)
        for (int t = tid; t < g.ntiles; t += bs) {
            const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + g.xoff;
#pragma unroll
                for (int cc = 0; cc < TILE; ++cc) {
                    const double sw = (double)w.swp[pp + cc];
                    w.Pb[pp + cc] = sw * sw * (double)w.dpad[pp + cc];
                }
            }
        }
        __syncthreads();
        const Conv64Gen<T, K> conv_ref{};
        conv_ref(w, g, 1);
        __syncthreads();
        double rs = 0;
        for (int i = tid; i < g.ns; i += bs) {
            const int ib = i / g.sx, ia = i - ib * g.sx;
            const double v = apply_LT_at<T, double, double>(g, w.E64, w.cst, w.Pc, ia, ib);
            rs += v * v;
        }
        const double rhsn = sqrt(block_sum(rs, red, which));
        which ^= 1;

        // ---- Jacobi preconditioner of the inner solves (see lwl_diag_at):
        // omega at every image pixel into Pa (free until the first residual;
        // sqrt(W) is zero in the padding frame), in FP32 like the inner solves
        for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {
            const int tile = t >> 4, q = t & 15;
            const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
            const int pp = (ty * TILE + (q >> 2) + g.hk) * g.Wp + tx * TILE + (q & 3) + g.xoff;
            float om = 0.f;
            for (int a = 0; a < g.K; ++a) {
                const T* srow = w.swp + pp + (a - g.hk) * g.Wp - g.hk;
                for (int b = 0; b < g.K; ++b) {
                    const float f = (float)P.psf[a * g.K + b], sv = (float)srow[b];
                    om = fmaf(f * f, sv * sv, om);
                }
            }
            w.Pa[pp] = (double)om;
        }
        __syncthreads();
        for (int i = tid; i < g.ns; i += bs) {
            const int ib = i / g.sx, ia = i - ib * g.sx;
            w.minv[i] = (T)1 / (lwl_diag_at<T>(g, w.E, w.cst, w.Pa, ia, ib) + (T)lam * hth_diag_at<T>(g, ia, ib));
        }
        __syncthreads();
        for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {  // Pa back to zero
            const int tile = t >> 4, q = t & 15;
            const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
            w.Pa[(ty * TILE + (q >> 2) + g.hk) * g.Wp + tx * TILE + (q & 3) + g.xoff] = 0.0;
        }

        // ---- starting point: the previous lambda of the chain, a given
        // warm start, or zero (the paper's blank source)
        if (ch.warm && ch.prev_ok) {
            // w.x64 still holds the previous lambda's solution
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
        // inner target: a 30x reduction per FP32 inner solve keeps each inner
        // solve short (FP32 loses orthogonality on long ones) at few FP64 passes
        const double eta_min = sizeof(T) == 4 ? A.eta : FINAL_MARGIN64 * A.tol;
        bool reverted = false;
        for (int outer = 0;; ++outer) {
            chi2 = residual64<T>(w, g, lam, red, which, reg2, g64, conv_ref);
            rel64 = rhsn > 0 ? sqrt(g64) / rhsn : 0.0;
            if (reverted) {  // the best iterate, evaluated again
                status |= ST_STAG;
                break;
            }
            if (outer > 0 && !(rel64 <= prev_rel)) {
                // the last correction raised the true residual (the inner
                // solve's operator is too coarse for this system at this
                // level): back to the best iterate; the next pass evaluates
                // it and stops
                for (int i = tid; i < g.ns; i += bs) w.x64[i] = w.xb[i];
                __syncthreads();
                reverted = true;
                continue;
            }
            if (!isfinite(rel64)) {
                status |= ST_BREAK;
                break;
            }
            if (!(rel64 > A.tol)) break;  // converged (or rhs = 0)
            if (total_it >= maxit || outer >= MAX_OUTER) {
                status |= ST_MAXIT;
                break;
            }
            // two refinement steps in a row that gain less than 10% each: stop
            slow = (outer > 0 && rel64 > 0.9 * prev_rel) ? slow + 1 : 0;
            if (slow >= 2) {
                status |= ST_STAG;
                break;
            }
            prev_rel = rel64;  // the residuals accepted so far decrease: this is the best iterate
            for (int i = tid; i < g.ns; i += bs) w.xb[i] = w.x64[i];
            // ---- inner solve of the correction equation A d = r: Jacobi-
            // preconditioned CG on the normal equations, from d = 0.  r (the
            // FP64 residual rounded to T) is the first gradient g (w.s); z =
            // M^-1 g lives in qreg and H p in rreg (both at least ns long).
            // Every vector of the recursion is of the size of the correction,
            // so rounding stays relative to it (an image-space CGLS residual
            // would carry the data misfit into every gradient).
            const double target =
                fmax(eta_min, fmin(MAX_TARGET, (sizeof(T) == 4 ? FINAL_MARGIN : FINAL_MARGIN64) * A.tol / rel64));
            for (int i = tid; i < g.ns; i += bs) {
                w.x[i] = 0;
                const T z = w.minv[i] * w.s[i];
                w.qreg[i] = z;
                w.p[i] = z;
            }
            {
                T gs = 0;
                for (int i = tid; i < g.ns; i += bs) gs = fma(w.s[i], w.qreg[i], gs);
                const double gam = block_sum_to0<T>(gs, red);
                if (tid == 0) {
                    ctl->gam = gam;
                    ctl->g0 = gam;
                    ctl->best = 1.0;
                    ctl->best_it = 0;
                    ctl->it = 0;
                    ctl->total_it = total_it;
                    ctl->brk = !isfinite(gam);
                    ctl->stop = ctl->brk || !(gam > 0.0) || total_it >= maxit;
                }
                __syncthreads();
            }
            const int stag_window = max(4000, 2 * g.ns);
            const T lamT = (T)lam;
            // per-cell L^T sums: bilinear and nearest only, when they fit in P2
            const bool cells_fit = g.interp != 2 && 4 * g.ncells <= g.plen;
            while (!ctl->stop) {
                // A p = L^T B^T W B L p + lam H^T H p: first L p and H p
                apply_L<T, T, T, T>(g, w.E, w.inv, w.p, w.P1);
                T dh = 0;
                for (int i = tid; i < g.nreg; i += bs) {
                    const T h = apply_H_row<T, T>(g, w.p, i);
                    w.rreg[i] = h;
                    dh = fma(h, h, dh);
                }
                __syncthreads();
                // q = sqrt(W) B L p; delta = p^T A p = ||q||^2 + lam ||H p||^2
                T cq;
                if constexpr (K == 0 && BIG)
                    cq = w.fft ? conv_pass_fft<T>(&w.fft->t, w.P1, w.swp, w.qimg, g, CONV_Q)
                               : conv_pass<T, K, SH>(w.P1, w.taps, w.swp, w.qimg, g, CONV_Q);
                else
                    cq = conv_pass<T, K, SH>(w.P1, w.taps, w.swp, w.qimg, g, CONV_Q);
                {
                    const double delta = block_sum_to0<T>(cq + lamT * dh, red);
                    if (tid == 0) {
                        if (!(delta > 0.0) || !isfinite(delta)) {
                            ctl->brk = 1;
                            ctl->stop = 1;
                        } else {
                            ctl->a_d = ctl->gam / delta;
                            ctl->a_f = (float)ctl->a_d;
                        }
                    }
                    __syncthreads();
                }
                if (ctl->brk) break;
                const T a = sizeof(T) == 4 ? (T)ctl->a_f : (T)ctl->a_d;
                // P2 = W B L p = sqrt(W) q
                for (int t = tid; t < g.ntiles; t += bs) {
                    const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
#pragma unroll
                    for (int r = 0; r < TILE; ++r) {
                        const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + g.xoff;
                        const V4<T> qv = ld4(w.qimg + pp), sw = ld4(w.swp + pp);
                        V4<T> o;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) o.v[cc] = sw.v[cc] * qv.v[cc];
                        st4(w.P2 + pp, o);
                    }
                }
                __syncthreads();  // P2 complete
                if constexpr (K == 0 && BIG) {
                    if (w.fft)
                        conv_pass_fft<T>(&w.fft->t, w.P2, nullptr, w.qimg, g, CONV_RAW);
                    else
                        conv_pass<T, K, SH>(w.P2, w.taps + g.K * g.kp, nullptr, w.qimg, g, CONV_RAW);
                } else {
                    conv_pass<T, K, SH>(w.P2, w.taps + g.K * g.kp, nullptr, w.qimg, g, CONV_RAW);
                }
                __syncthreads();  // u complete
                // (A p)_i = (L^T u)_i + lam (H^T H p)_i, then the CG updates of
                // x, g (w.s) and z = M^-1 g (w.qreg)
                T gs = 0;
                if (cells_fit) {
                    // L^T u in two passes: per cell, the four corner sums of its
                    // rays (each ray read once) into P2's storage (free until the
                    // next W B L p store); then per source pixel the fixed-order
                    // sum of the corners it receives from its (up to) four cells
                    T* cp = w.P2;
                    for (int cell = tid; cell < g.ncells; cell += bs) {
                        const int k1 = w.cst[cell + 1];
                        T c00 = 0, c10 = 0, c01 = 0, c11 = 0;
                        for (int k = w.cst[cell]; k < k1; ++k) {
                            const Entry<T> en = w.E[k];
                            const T U = w.qimg[en.ppos];
                            const T uU = en.u * U, u0 = U - uU;  // u U, (1-u) U
                            c00 = fma((T)1 - en.v, u0, c00);
                            c10 = fma((T)1 - en.v, uU, c10);
                            c01 = fma(en.v, u0, c01);
                            c11 = fma(en.v, uU, c11);
                        }
                        cp[4 * cell + 0] = c00;
                        cp[4 * cell + 1] = c10;
                        cp[4 * cell + 2] = c01;
                        cp[4 * cell + 3] = c11;
                    }
                    __syncthreads();
                    for (int i = tid; i < g.ns; i += bs) {
                        const int ib = i / g.sx, ia = i - ib * g.sx;
                        T acc = 0;
                        if (ib <= g.sy - 2 && ia <= g.sx - 2) acc += cp[4 * (ib * g.ncx + ia) + 0];
                        if (ib <= g.sy - 2 && ia >= 1) acc += cp[4 * (ib * g.ncx + ia - 1) + 1];
                        if (ib >= 1 && ia <= g.sx - 2) acc += cp[4 * ((ib - 1) * g.ncx + ia) + 2];
                        if (ib >= 1 && ia >= 1) acc += cp[4 * ((ib - 1) * g.ncx + ia - 1) + 3];
                        const T ap = acc * g.invNp + lamT * apply_HT_at<T, T>(g, w.rreg, i, ia, ib);
                        w.x[i] = fma(a, w.p[i], w.x[i]);
                        const T gv = fma(-a, ap, w.s[i]);
                        const T z = w.minv[i] * gv;
                        w.s[i] = gv;
                        w.qreg[i] = z;
                        gs = fma(gv, z, gs);
                    }
                } else {
                    for (int i = tid; i < g.ns; i += bs) {
                        const int ib = i / g.sx, ia = i - ib * g.sx;
                        const T ap = apply_LT_at<T, T, T>(g, w.E, w.cst, w.qimg, ia, ib) +
                                     lamT * apply_HT_at<T, T>(g, w.rreg, i, ia, ib);
                        w.x[i] = fma(a, w.p[i], w.x[i]);
                        const T gv = fma(-a, ap, w.s[i]);
                        const T z = w.minv[i] * gv;
                        w.s[i] = gv;
                        w.qreg[i] = z;
                        gs = fma(gv, z, gs);
                    }
                }
                {
                    const double gnew = block_sum_to0<T>(gs, red);
                    if (tid == 0) {
                        ctl->b_d = gnew / ctl->gam;
                        ctl->b_f = (float)ctl->b_d;
                        ctl->gam = gnew;
                        const int it = ++ctl->it;
                        ++ctl->total_it;
                        const double rel = sqrt(gnew / ctl->g0);
                        if (!isfinite(gnew)) {
                            ctl->brk = 1;
                            ctl->stop = 1;
                        } else if (!(rel > target) || ctl->total_it >= maxit) {
                            ctl->stop = 1;
                        } else if (rel < 0.5 * ctl->best) {
                            ctl->best = rel;
                            ctl->best_it = it;
                        } else if (it - ctl->best_it > stag_window) {
                            ctl->stop = 1;
                        }
                    }
                    __syncthreads();
                }
                // the cell sums overwrote part of P2's zero frame: clear them
                if (cells_fit)
                    for (int i = tid; i < 4 * g.ncells; i += bs) w.P2[i] = 0;
                const T bt = sizeof(T) == 4 ? (T)ctl->b_f : (T)ctl->b_d;
                for (int i = tid; i < g.ns; i += bs) w.p[i] = fma(bt, w.p[i], w.qreg[i]);
                __syncthreads();
            }
            total_it = ctl->total_it;
            if (ctl->brk) status |= ST_BREAK;
            if (status & ST_BREAK) break;
            for (int i = tid; i < g.ns; i += bs) w.x64[i] += (double)w.x[i];
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
        ch.prev_ok = !(status & ST_BREAK);
    }
}

// ---------------------------------------------------------------------------
// k_finalize: L-curve corner per candidate (Section 2.6), status, s_out
// ---------------------------------------------------------------------------
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
// k_forward: model = B L s and Eq. chi2 for a batch of sources at one lens
// (candidate scratch of index 0).  One CTA per source (grid-stride); the
// L s image lives in a per-CTA global slab.
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(NTHREADS, 1) k_forward(const Prob<T>* __restrict__ probs, CandScratch<T> cs,
                                                         const T* __restrict__ S, int n_src, T* model,
                                                         double* chi2, T* slab, long long slab_stride,
                                                         int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob<T>& P = probs[0];
    const Geo<T> g = geo_of(P, cs.nent[0]);
    double* red = reinterpret_cast<double*>(smem + 16);
    T* taps = reinterpret_cast<T*>(smem + 16 + 2 * 33 * sizeof(double));
    Work<T> w;
    w.E = cs.E;
    w.inv = cs.inv;
    w.cst = cs.cst;
    T* P1 = slab + (long long)blockIdx.x * slab_stride;
    const int tid = threadIdx.x;
    for (int i = tid; i < g.K * g.kp; i += blockDim.x) {
        const int a = i / g.kp, b = i - a * g.kp;
        taps[i] = b < g.K ? P.psf[(g.K - 1 - a) * g.K + (g.K - 1 - b)] : (T)0;
    }
    for (int i = tid; i < g.plen; i += blockDim.x) P1[i] = 0;
    if (blockIdx.x == 0 && tid == 0 && status) status[0] = cs.cstat[0];
    int which = 0;
    const bool bad = (cs.cstat[0] & ST_BADPARAM) != 0;
    for (int k = blockIdx.x; k < n_src; k += gridDim.x) {
        __syncthreads();
        if (bad) {
            if (tid == 0) chi2[k] = __longlong_as_double(0x7ff0000000000000LL);
            continue;
        }
        apply_L<T, T, T, T>(g, w.E, w.inv, S + (long long)k * g.ns, P1);
        __syncthreads();
        double chi = 0;
        for (int t = tid; t < g.ntiles; t += blockDim.x) {
            const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
            T acc[TILE][TILE];
            const T* base = P1 + (ty * TILE) * g.Wp + tx * TILE;
            if constexpr (K > 0)
                conv_tile<T, K, false>(base, g.Wp, taps, acc);
            else
                conv_tile_rt<T, T>(base, g.Wp, taps, g.K, g.kp, g.sh, acc);
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                const int y = ty * TILE + r;
                const int pp = (y + g.hk) * g.Wp + tx * TILE + g.xoff;
#pragma unroll
                for (int cc = 0; cc < TILE; ++cc) {
                    const int x = tx * TILE + cc;
                    const double sw = (double)cs.swp[pp + cc];
                    const double res = sw * ((double)cs.dpad[pp + cc] - (double)acc[r][cc]);
                    chi += res * res;
                    if (model && y < g.ny && x < g.nx) model[(long long)k * g.nx * g.ny + y * g.nx + x] = acc[r][cc];
                }
            }
        }
        const double cval = block_sum(chi, red, which);
        which ^= 1;
        if (tid == 0) chi2[k] = cval;
    }
}

// PSF spectra of the problems that convolve by FFT, one CTA per problem:
// the FP64 spectrum (fft_psf_spectrum) and, for FP32 contexts, its rounding
// to float.  Problems with fft_m == 0 are skipped.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_psf_spectra(const Prob<T>* __restrict__ probs, double2* spec64,
                                                        float2* spec32, long long stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob<T>& P = probs[blockIdx.x];
    if (P.fft_m == 0) return;
    const int M = P.fft_m;
    double2* tw = reinterpret_cast<double2*>(smem);
    FftPlan<double> f;
    f.M = M;
    f.logM = P.fft_log;
    f.nb = fft_batch_count<double2>(M);
    f.tw = tw;
    f.b0 = reinterpret_cast<double2*>(smem + align_up<T>(sizeof(double2) * (M - 1), 16));
    f.b1 = f.b0 + f.nb * (M + 1);
    f.F = spec64 + (long long)blockIdx.x * stride;
    fft_twiddles<double>(tw, M);
    __syncthreads();
    fft_psf_spectrum<double>(f, P.psf, P.K);
    if (spec32) {
        const int n = ((M >> 1) + 1) * M;
        float2* o = spec32 + (long long)blockIdx.x * stride;
        for (int i = threadIdx.x; i < n; i += blockDim.x) o[i] = make_float2((float)f.F[i].x, (float)f.F[i].y);
    }
}

}  // namespace mirage
