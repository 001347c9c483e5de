// Fast-path CGLS item kernel for small images (FP32 contexts).
//
// Same method as k_cgls (FP32 inner CGLS inside the FP64 residual
// refinement), laid out for two resident CTAs per SM:
//   * one ray per pixel and an identity or Laplacian H (square H);
//   * each thread owns exactly one 4x4 image tile (images up to 256 tiles)
//     and keeps that tile's residual, sqrt(W), q = sqrt(W) B L p and mapped
//     mask in registers; each thread also owns up to NSP source pixels
//     (i = tid + k * blockDim.x) and keeps their x, s and sqrt(lam) H p;
//   * shared memory holds only the two padded convolution buffers (P1 = L p,
//     reused for u = B^T sqrt(W) r at mapped pixels; P2 = sqrt(W) r, reused
//     for the per-cell partial sums of L^T u), the rays in 12-byte form,
//     16-bit cell starts, p and r_reg;
//   * the convolution uses packed FP32x2 FMAs (__ffma2_rn) on tap pairs
//     stored duplicated in shared memory.
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

// tap source of the fast convolution
enum : int { TAPS_SMEM_X2 = 0, TAPS_PARAM = 1, TAPS_PARAM_X2 = 2 };

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
#pragma unroll
            for (int b = 0; b < K; ++b) {
                const int o = b + SHF;
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const int a = i - r;
                    if (a >= 0 && a < K) {
                        const float t = pt[a * K + b];
                        if constexpr (MODE == TAPS_PARAM) {
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
            if constexpr (MODE == TAPS_PARAM) {
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

template <int K, int NSP, int MODE>
__global__ void __launch_bounds__(NTHREADS, 2) k_cgls_fast(const __grid_constant__ FastArgs FA) {
    using T = float;
    const CglsArgs<float>& A = FA.A;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, bs = blockDim.x;
    int* slot = reinterpret_cast<int*>(smem);
    double* red = reinterpret_cast<double*>(smem + 16);
    CgCtl* ctl = reinterpret_cast<CgCtl*>(smem + 16 + 2 * 33 * sizeof(double));
    float* pbuf = reinterpret_cast<float*>(red);  // 2 x 32 float2 for block_pair_all
    int last_c = -1;
    int which = 0;
    // per-phase clocks (thread 0): 0 L p + H p, 1 B conv + reduce, 2 updates,
    // 3 B^T conv, 4 L^T + reduce + p, 5 FP64 refinement, 6 item setup
    unsigned long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool timed = A.phase_clk != nullptr && threadIdx.x == 0;
    unsigned long long t_last = timed ? clock64() : 0ull;
#define PHASE(n)                                  \
    do {                                          \
        if (timed) {                              \
            const unsigned long long t_ = clock64(); \
            ph[n] += t_ - t_last;                 \
            t_last = t_;                          \
        }                                         \
    } while (0)

    while (true) {
        __syncthreads();
        if (tid == 0) slot[0] = atomicAdd(A.counter, 1);
        __syncthreads();
        const int it_idx = slot[0];
        if (it_idx >= A.n_items) break;
        const int packed = A.items[it_idx];
        const int c = packed / MAX_LAM, k = packed - c * MAX_LAM;
        const Prob<T>& P = A.probs[A.cand_prob[c]];
        const CandScratch<T>& cs = A.cs;
        const int nent = cs.nent[c];
        const Geo<T> g = geo_of(P, nent);

        // ---- carve shared memory
        unsigned char* sp = smem + 16 + 2 * 33 * sizeof(double) + 128;
        float2* taps2 = reinterpret_cast<float2*>(sp);
        sp += align_up<T>(sizeof(float2) * 2 * K * K, 16);
        Work<T> w;
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
        __syncthreads();

        // ---- tile ownership, sqrt(W) and mapped mask in registers
        const bool own = tid < g.ntiles;
        const int ty = own ? tid / g.tiles_x : 0, tx = own ? tid - (tid / g.tiles_x) * g.tiles_x : 0;
        const int pp0 = (ty * TILE + g.hk) * g.Wp + tx * TILE + g.xoff;
        const float* P1t = P1 + (ty * TILE) * g.Wp + tx * TILE;
        const float* P2t = P2 + (ty * TILE) * g.Wp + tx * TILE;
        float sw[16], rr[16];
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
            continue;
        }

        const double lam = A.lambdas[(long long)c * A.max_lam + k];
        const float sl = (float)sqrt(lam);
        const int maxit = A.maxit > 0 ? A.maxit : 25 * g.ns;
        PHASE(6);

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
        conv64_pass<T>(w, g, 1);
        __syncthreads();
        double rs = 0;
        for (int i = tid; i < g.ns; i += bs) {
            const int ib = i / g.sx, ia = i - ib * g.sx;
            const double v = apply_LT_at<T, double, double>(g, w.E64, w.cst, w.Pc, ia, ib);
            rs += v * v;
        }
        const double rhsn = sqrt(block_sum(rs, red, which));
        which ^= 1;

        // ---- Jacobi preconditioner of the inner solves: an approximation of
        // diag(A~^T A~) = diag(L^T B^T W B L) + lam diag(H^T H), taking
        // diag(L^T B^T W B L)_i ~ sum_rays weight_i^2 w_pixel * sum(psf^2)
        // (exact for a delta PSF; cross terms between rays are dropped).
        // Any positive diagonal leaves the solution unchanged; this one cuts
        // the CGLS iterations two- to threefold.
        float minv[NSP];
        {
            if (tid < 32) {
                float a = 0.f;
                for (int i = tid; i < K * K; i += 32) a = fmaf(P.psf[i], P.psf[i], a);
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (tid == 0) reinterpret_cast<float*>(ctl)[0] = a;
            }
            float4* cellp = reinterpret_cast<float4*>(P2);
            for (int cell = tid; cell < g.ncells; cell += bs) {
                const int k0 = cst16[cell], k1 = cst16[cell + 1];
                float c00 = 0.f, c10 = 0.f, c01 = 0.f, c11 = 0.f;
                for (int e = k0; e < k1; ++e) {
                    const unsigned id = eidx[e];
                    const float2 uv = euv[e];
                    const float sw1 = w.swp[id & 0xffffu];
                    const float W2 = sw1 * sw1;
                    const float u1 = uv.x * uv.x, u0 = (1.f - uv.x) * (1.f - uv.x);
                    const float v1 = uv.y * uv.y, v0 = (1.f - uv.y) * (1.f - uv.y);
                    c00 = fmaf(u0 * v0, W2, c00);
                    c10 = fmaf(u1 * v0, W2, c10);
                    c01 = fmaf(u0 * v1, W2, c01);
                    c11 = fmaf(u1 * v1, W2, c11);
                }
                cellp[cell] = make_float4(c00, c10, c01, c11);
            }
            __syncthreads();
            const float psf2 = reinterpret_cast<const float*>(ctl)[0];
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
                    minv[kk] = 1.f / (dsum * psf2 + (float)lam * h);
                }
            }
            __syncthreads();
            for (int cell = tid; cell < g.ncells; cell += bs) cellp[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
        }

        if (A.warm_x) {
            const T* x0 = A.warm_x + ok * A.max_ns;
            for (int i = tid; i < g.ns; i += bs) w.x64[i] = (double)x0[i];
        } else {
            for (int i = tid; i < g.ns; i += bs) w.x64[i] = 0.0;
        }
        __syncthreads();

        int status = 0, total_it = 0, slow = 0;
        double chi2 = 0, reg2 = 0, g64 = 0, rel64 = 0, prev_rel = 1e300;
        constexpr int MAX_OUTER = 16;
        const double eta_min = 0.03;
        for (int outer = 0;; ++outer) {
            PHASE(6);
            chi2 = residual64<T>(w, g, lam, red, which, reg2, g64);
            PHASE(5);
            rel64 = rhsn > 0 ? sqrt(g64) / rhsn : 0.0;
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
            prev_rel = rel64;
            const double target = fmax(eta_min, 0.3 * A.tol / rel64);

            // ---- inner CGLS on the correction: state into registers
            float x[NSP], s[NSP], qr[NSP];
            float gs = 0.f;
#pragma unroll
            for (int kk = 0; kk < NSP; ++kk) {
                const int i = tid + kk * bs;
                x[kk] = 0.f;
                s[kk] = 0.f;
                if (i < g.ns) {
                    s[kk] = w.s[i];
                    const float z = minv[kk] * s[kk];
                    p[i] = z;
                    gs = fmaf(s[kk], z, gs);
                }
            }
            if (own) {
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const V4<float> r4 = ld4(w.rimg + pp0 + r * g.Wp);
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) rr[r * 4 + cc] = r4.v[cc];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) rr[q] = 0.f;
            }
            int half = 0, it_in = 0, best_it = 0, brk = 0, stop = 0;
            float gam, g0, best = 1.f;
            {
                const float2 gp = block_pair_all(gs, pbuf, half);
                half ^= 1;
                gam = gp.x + gp.y;
                g0 = gam;
                brk = !isfinite(gam);
                stop = brk || !(gam > 0.f) || total_it >= maxit;
            }
            const int stag_window = max(4000, 2 * g.ns);
            while (!stop) {
                // P1 <- L p at the mapped pixels; q_reg = sqrt(lam) H p
                for (int e = tid; e < nent; e += bs) {
                    const unsigned id = eidx[e];
                    const float2 uv = euv[e];
                    const float* s0 = p + (id >> 16);
                    P1[id & 0xffffu] = (1.f - uv.y) * ((1.f - uv.x) * s0[0] + uv.x * s0[1]) +
                                       uv.y * ((1.f - uv.x) * s0[g.sx] + uv.x * s0[g.sx + 1]);
                }
                float dq = 0.f;
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    qr[kk] = 0.f;
                    if (i < g.ns) {
                        qr[kk] = sl * apply_H_row<T, float>(g, p, i);
                        dq = fmaf(qr[kk], qr[kk], dq);
                    }
                }
                __syncthreads();
                PHASE(0);
                // q = sqrt(W) B P1 on the owned tile
                float q[16];
                if (own) {
                    float o16[16];
                    conv_tile_fast<K, MODE>(P1t, g.Wp, taps2, FA.ptap[0], o16);
#pragma unroll
                    for (int qq = 0; qq < 16; ++qq) q[qq] = sw[qq] * o16[qq];
#pragma unroll
                    for (int qq = 0; qq < 16; ++qq) dq = fmaf(q[qq], q[qq], dq);
                } else {
#pragma unroll
                    for (int qq = 0; qq < 16; ++qq) q[qq] = 0.f;
                }
                const float2 dl = block_pair_all(dq, pbuf, half);
                half ^= 1;
                const float delta = dl.x + dl.y;
                PHASE(1);
                if (!(delta > 0.f) || !isfinite(delta)) {
                    brk = 1;
                    break;
                }
                const float a = gam / delta;
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    if (i < g.ns) {
                        x[kk] = fmaf(a, p[i], x[kk]);
                        rreg[i] = fmaf(-a, qr[kk], rreg[i]);
                    }
                }
                if (own) {
#pragma unroll
                    for (int r = 0; r < TILE; ++r) {
                        V4<float> o;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            rr[r * 4 + cc] = fmaf(-a, q[r * 4 + cc], rr[r * 4 + cc]);
                            o.v[cc] = sw[r * 4 + cc] * rr[r * 4 + cc];
                        }
                        st4(P2 + pp0 + r * g.Wp, o);
                    }
                }
                __syncthreads();  // P2 complete
                PHASE(2);
                // u = B^T P2 on the owned tile, stored into P1 at mapped pixels
                if (own) {
                    float o16[16];
                    conv_tile_fast<K, MODE>(P2t, g.Wp, taps2 + K * K, FA.ptap[1], o16);
#pragma unroll
                    for (int r = 0; r < TILE; ++r) {
                        float* dst = P1 + pp0 + r * g.Wp;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            if (mbits & (1u << (r * 4 + cc))) dst[cc] = o16[r * 4 + cc];
                    }
                }
                __syncthreads();  // u complete
                PHASE(3);
                // L^T u in two passes (deterministic): per cell, the four corner
                // sums of its rays (each ray read once), kept in P2's storage;
                // then per source pixel, the fixed-order sum of the corners
                // it receives from its (up to) four cells
                float4* cellp = reinterpret_cast<float4*>(P2);
                for (int cell = tid; cell < g.ncells; cell += bs) {
                    const int k0 = cst16[cell], k1 = cst16[cell + 1];
                    float c00 = 0.f, c10 = 0.f, c01 = 0.f, c11 = 0.f;
#pragma unroll 2
                    for (int e = k0; e < k1; ++e) {
                        const unsigned id = eidx[e];
                        const float2 uv = euv[e];
                        const float U = P1[id & 0xffffu];
                        const float uU = uv.x * U, u0 = U - uU;  // u U, (1-u) U
                        c00 = fmaf(1.f - uv.y, u0, c00);
                        c10 = fmaf(1.f - uv.y, uU, c10);
                        c01 = fmaf(uv.y, u0, c01);
                        c11 = fmaf(uv.y, uU, c11);
                    }
                    cellp[cell] = make_float4(c00, c10, c01, c11);
                }
                __syncthreads();
                PHASE(7);
                float gsum = 0.f;
#pragma unroll
                for (int kk = 0; kk < NSP; ++kk) {
                    const int i = tid + kk * bs;
                    if (i < g.ns) {
                        const int ib = i / g.sx, ia = i - ib * g.sx;
                        const float* cp = reinterpret_cast<const float*>(cellp);
                        float acc = 0.f;
                        // (dx, dy) = position of i in the cell: component dx + 2 dy
                        if (ib <= g.sy - 2 && ia <= g.sx - 2) acc += cp[4 * (ib * g.ncx + ia) + 0];
                        if (ib <= g.sy - 2 && ia >= 1) acc += cp[4 * (ib * g.ncx + ia - 1) + 1];
                        if (ib >= 1 && ia <= g.sx - 2) acc += cp[4 * ((ib - 1) * g.ncx + ia) + 2];
                        if (ib >= 1 && ia >= 1) acc += cp[4 * ((ib - 1) * g.ncx + ia - 1) + 3];
                        const float gr = acc + sl * apply_HT_at<T, float>(g, rreg, i, ia, ib);
                        s[kk] = minv[kk] * gr;  // preconditioned gradient z = M^-1 g
                        gsum = fmaf(gr, s[kk], gsum);
                    }
                }
                const float2 gp = block_pair_all(gsum, pbuf, half);
                half ^= 1;
                const float gnew = gp.x + gp.y;
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
                    if (i < g.ns) p[i] = fmaf(bt, p[i], s[kk]);
                }
                // the cell partials overwrote P2's zero frame: clear them
                for (int cell = tid; cell < g.ncells; cell += bs) cellp[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncthreads();
                PHASE(4);
            }
            if (brk) {
                status |= ST_BREAK;
                break;
            }
#pragma unroll
            for (int kk = 0; kk < NSP; ++kk) {
                const int i = tid + kk * bs;
                if (i < g.ns) w.x64[i] += (double)x[kk];
            }
            // the inner loop leaves u in P1 at mapped pixels: restore zeros
            // there is not needed (L p overwrites every mapped pixel)
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
    }
    if (timed)
        for (int i = 0; i < 8; ++i) atomicAdd(A.phase_clk + i, ph[i]);
#undef PHASE
}

// shared memory of the fast variant (0 if the problem is not eligible)
__host__ inline size_t fast_smem_bytes(const Prob<float>& P) {
    if (P.Np != 1 || P.ntiles > NTHREADS || P.plen >= 65536 || P.nrays >= 65536 || P.ns >= 65536 ||
        P.nreg != P.ns || 4 * P.ncells > P.plen)
        return 0;
    size_t o = 16 + 2 * 33 * sizeof(double) + 128;
    o += align_up<float>(sizeof(float2) * 2 * P.K * P.K, 16);
    o += align_up<float>(sizeof(double) * 2 * P.K * P.kp, 16);
    o += 2 * align_up<float>(sizeof(float) * P.plen, 16);
    o += align_up<float>(sizeof(unsigned) * (size_t)P.nrays, 16);
    o += align_up<float>(sizeof(float2) * (size_t)P.nrays, 16);
    o += align_up<float>(sizeof(unsigned short) * (size_t)(P.ncells + 1), 16);
    o += align_up<float>(sizeof(float) * P.ns, 16);
    o += align_up<float>(sizeof(float) * P.nreg, 16);
    return o;
}

__host__ inline size_t fast_slab_bytes(const Prob<float>& P) {
    size_t o = sizeof(double) * (3 * align_up<float>(P.plen, 4) + align_up<float>(P.ns, 4) + align_up<float>(P.nreg, 4));
    o += sizeof(float) * (align_up<float>(P.plen, 4) + align_up<float>(P.ns, 4));
    return align_up<float>(o, 256);
}

}  // namespace mirage
