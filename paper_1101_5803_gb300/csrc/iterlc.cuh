// Fixed-iteration CGLS with the L-curve over the iterations (Section 2.6)
// and the Monte Carlo estimate of the degrees of freedom (Section 2.5).
//
// The paper's own inner loop: CGLS (Section 2.4) on the weighted
// least-squares problem min ||sqrt(W)(B L s - d)|| from a blank source, for
// a fixed number of iterations; the iteration count is the regulariser.
// After every iteration k the kernel records the image chi^2 of s_k (the
// squared norm of the CGLS residual) and the zeroth-order regularisation
// measure sum s_k^2; the L-curve through (log10 sum s_k^2, log10 chi^2_k)
// gives the corner iteration, whose chi^2 is the candidate's fitness and
// whose source is returned.  With a Gaussian image bhat, a twin CGLS on
// m * bhat driven by the same step coefficients alpha_k, beta_k yields
// dof_k = bhat^T (bhat - A xhat_k), the trace estimate of the residual's
// degrees of freedom (reduced chi^2 = chi^2_k / dof_k).
//
// The iteration runs in FP64 in every context: without a regulariser CGLS
// loses orthogonality within a few iterations on these problems, and from
// then on its trajectory (hence the L-curve and its corner) depends on the
// rounding; in FP32 it leaves the exact-arithmetic path within ten
// iterations, in FP64 it stays on it to 1e-14 through the corner.  FP32
// contexts read their FP32 image data and the ray trace's FP64 weights.
//
// One CTA per candidate (persistent over the candidates); every vector in
// the CTA's global slab (L2-resident), the taps in shared memory.  The
// iterates are kept in the slab so that the corner's source can be copied
// out after the corner is known.
#pragma once

#include "kernels.cuh"

namespace mirage {

template <typename T>
struct IterArgs {
    const Prob<T>* probs;
    const int* cand_prob;   // [n_cand]
    CandScratch<T> cs;      // ray-trace output
    int n_cand, n_iter, max_ns;
    const T* bhat;          // nullable [n_probs][bhat_stride] unpadded images (row-major, y slow)
    long long bhat_stride;
    int* counter;           // candidate queue
    void* slab;
    long long slab_stride;  // bytes per CTA
    double* chi2;           // [n_cand][n_iter + 1]
    double* reg;            // [n_cand][n_iter + 1] sum s_k^2
    double* dof;            // nullable [n_cand][n_iter + 1]
    double* kappa;          // nullable [n_cand][n_iter + 1]
    int* corner;            // [n_cand] corner iteration (1..n_iter)
    T* s_out;               // nullable [n_cand][max_ns]
    int* status;            // [n_cand]
};

// shared memory of k_cgls_iter (FP64 taps)
template <typename T>
__host__ __device__ inline size_t iter_smem_bytes(int K, int kp) {
    return 16 + (2 * 33 + MAX_LAM + 2) * sizeof(double) + align_up<T>(sizeof(double) * 2 * K * kp, 16);
}

// per-CTA slab of k_cgls_iter (FP64): sqrt(W), rimg, qimg, P1, P2, rhat
// (images); x, p, s, xhat, phat, shat (source vectors); the n_iter + 1 iterates
template <typename T>
__host__ inline size_t iter_slab_bytes(const Prob<T>& P, int n_iter) {
    const size_t pl = align_up<T>(P.plen, 4), pn = align_up<T>(P.ns, 4);
    return align_up<T>(sizeof(double) * (6 * pl + 6 * pn + (size_t)(n_iter + 1) * pn), 256);
}

// the geometry with FP64 interpolation weights
template <typename T>
__device__ __forceinline__ Geo<double> geo_fp64(const Geo<T>& g) {
    Geo<double> d;
    d.nx = g.nx;
    d.ny = g.ny;
    d.sx = g.sx;
    d.sy = g.sy;
    d.ns = g.ns;
    d.nreg = g.nreg;
    d.K = g.K;
    d.hk = g.hk;
    d.kp = g.kp;
    d.xoff = g.xoff;
    d.sh = g.sh;
    d.Np = g.Np;
    d.ncx = g.ncx;
    d.ncells = g.ncells;
    d.Wp = g.Wp;
    d.plen = g.plen;
    d.tiles_x = g.tiles_x;
    d.ntiles = g.ntiles;
    d.reg = g.reg;
    d.nent = g.nent;
    d.interp = g.interp;
    d.invNp = (double)g.invNp;
    return d;
}

template <typename T, int K>
__global__ void __launch_bounds__(NTHREADS) k_cgls_iter(IterArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, bs = blockDim.x;
    int* slot = reinterpret_cast<int*>(smem);
    double* red = reinterpret_cast<double*>(smem + 16);
    double* kap = red + 2 * 33;  // [MAX_LAM] curvature scratch of the corner pick
    double* taps = reinterpret_cast<double*>(smem + 16 + (2 * 33 + MAX_LAM + 2) * sizeof(double));
    int which = 0;
    const int n1 = A.n_iter + 1;

    while (true) {
        __syncthreads();
        if (tid == 0) slot[0] = atomicAdd(A.counter, 1);
        __syncthreads();
        const int c = slot[0];
        if (c >= A.n_cand) break;
        const int pidx = A.cand_prob[c];
        const Prob<T>& P = A.probs[pidx];
        const CandScratch<T>& cs = A.cs;
        const int nent = cs.nent[c];
        const Geo<double> g = geo_fp64(geo_of(P, nent));
        double* chi2 = A.chi2 + (long long)c * n1;
        double* reg = A.reg + (long long)c * n1;
        double* dof = A.dof ? A.dof + (long long)c * n1 : nullptr;
        const bool twin = A.bhat != nullptr && dof != nullptr;
        const int cstat = cs.cstat[c];
        if (cstat & (ST_BADPARAM | ST_EMPTY)) {
            if (tid == 0) {
                for (int k = 0; k < n1; ++k) {
                    chi2[k] = (cstat & ST_BADPARAM) ? __longlong_as_double(0x7ff0000000000000LL) : 0.0;
                    reg[k] = 0.0;
                    if (dof) dof[k] = 0.0;
                    if (A.kappa) A.kappa[(long long)c * n1 + k] = 0.0;
                }
                A.corner[c] = 0;
                A.status[c] = cstat;
            }
            if (A.s_out)
                for (int i = tid; i < A.max_ns; i += bs) A.s_out[(long long)c * A.max_ns + i] = (T)0;
            continue;
        }

        // ---- buffers (FP64)
        const size_t pl = align_up<T>(g.plen, 4), pn = align_up<T>(g.ns, 4);
        double* ts = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(A.slab) + (long long)blockIdx.x * A.slab_stride);
        Work<double> w{};
        w.swp = ts; ts += pl;
        w.rimg = ts; ts += pl;
        w.qimg = ts; ts += pl;
        w.P1 = ts; ts += pl;
        w.P2 = ts; ts += pl;
        double* rh = ts; ts += pl;
        w.x = ts; ts += pn;
        w.p = ts; ts += pn;
        w.s = ts; ts += pn;
        double* xh = ts; ts += pn;
        double* ph = ts; ts += pn;
        double* sh = ts; ts += pn;
        double* iters_x = ts;  // [n1][pn]
        const T* g_swp = cs.swp + (long long)c * cs.sPad;
        const T* g_d = cs.dpad + (long long)c * cs.sPad;
        w.E = cs.E64 + (long long)c * cs.sE;  // FP64 weights (the ray trace's own, in both precisions)
        w.inv = cs.inv + (long long)c * cs.sInv;
        w.cst = cs.cst + (long long)c * cs.sCst;
        w.taps = taps;
        const T* bh = twin ? A.bhat + (long long)pidx * A.bhat_stride : nullptr;

        // taps: [0] flipped PSF for B, [1] PSF for B^T; rows padded to kp
        for (int i = tid; i < 2 * g.K * g.kp; i += bs) {
            const int h = i / (g.K * g.kp), rem = i - h * g.K * g.kp;
            const int a = rem / g.kp, b = rem - a * g.kp;
            double v = 0;
            if (b < g.K) v = h == 0 ? (double)P.psf[(g.K - 1 - a) * g.K + (g.K - 1 - b)] : (double)P.psf[a * g.K + b];
            taps[i] = v;
        }
        for (int i = tid; i < g.plen; i += bs) {
            w.swp[i] = (double)g_swp[i];  // sqrt(W), zero in the padding frame
            w.rimg[i] = 0;
            w.qimg[i] = 0;
            w.P1[i] = 0;
            w.P2[i] = 0;
            rh[i] = 0;
        }
        __syncthreads();
        // r_0 = sqrt(W) d (the weighted data); the twin's r_0 = m * bhat
        double c0 = 0.0, d0 = 0.0;
        for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {
            const int tile = t >> 4, q = t & 15;
            const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
            const int y = ty * TILE + (q >> 2), x = tx * TILE + (q & 3);
            const int pp = (y + g.hk) * g.Wp + x + g.xoff;
            const double r0 = (double)g_swp[pp] * (double)g_d[pp];
            w.rimg[pp] = r0;
            c0 += r0 * r0;
            if (twin && x < g.nx && y < g.ny && g_swp[pp] > (T)0) {
                const double b0 = (double)bh[y * g.nx + x];
                rh[pp] = b0;
                d0 += b0 * b0;
            }
        }
        c0 = block_sum(c0, red, which);
        which ^= 1;
        if (twin) {
            d0 = block_sum(d0, red, which);
            which ^= 1;
        }

        // A^T v for an image vector v (at tile positions): into dst, returns
        // the thread's partial sum of dst^2
        auto apply_AT = [&](const double* v, double* dst) -> double {
            for (int t = tid; t < g.ntiles; t += bs) {
                const int ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const int pp = (ty * TILE + r + g.hk) * g.Wp + tx * TILE + g.xoff;
                    const V4<double> rv = ld4(v + pp), sw = ld4(w.swp + pp);
                    V4<double> o;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) o.v[cc] = sw.v[cc] * rv.v[cc];
                    st4(w.P2 + pp, o);
                }
            }
            __syncthreads();
            conv_pass<double, K, false>(w.P2, taps + g.K * g.kp, nullptr, w.qimg, g, CONV_RAW);
            __syncthreads();
            double ss = 0.0;
            for (int i = tid; i < g.ns; i += bs) {
                const int ib = i / g.sx, ia = i - ib * g.sx;
                const double u = apply_LT_at<double, double, double>(g, w.E, w.cst, w.qimg, ia, ib);
                dst[i] = u;
                ss += u * u;
            }
            __syncthreads();
            return ss;
        };
        // q = A v into qimg (tile positions), returns the thread's partial sum of q^2
        auto apply_A = [&](const double* v) -> double {
            apply_L<double, double, double, double>(g, w.E, w.inv, v, w.P1);
            __syncthreads();
            const double ss = conv_pass<double, K, false>(w.P1, taps, w.swp, w.qimg, g, CONV_Q);
            __syncthreads();
            return ss;
        };

        // s_0 = A^T r_0, p_0 = s_0, x_0 = 0 (and the same for the twin)
        double gam = block_sum(apply_AT(w.rimg, w.s), red, which);
        which ^= 1;
        if (twin) apply_AT(rh, sh);
        for (int i = tid; i < g.ns; i += bs) {
            w.x[i] = 0;
            w.p[i] = w.s[i];
            iters_x[i] = 0;
            if (twin) {
                xh[i] = 0;
                ph[i] = sh[i];
            }
        }
        if (tid == 0) {
            chi2[0] = c0;
            reg[0] = 0.0;
            if (dof) dof[0] = twin ? d0 : 0.0;
        }
        __syncthreads();

        int done = 0, brk = 0;
        for (int k = 1; k <= A.n_iter; ++k) {
            if (!(gam > 0.0) || !isfinite(gam)) {  // exact fit (or breakdown): nothing left to do
                brk = !isfinite(gam);
                break;
            }
            // q = A p, alpha = gamma / ||q||^2
            const double delta = block_sum(apply_A(w.p), red, which);
            which ^= 1;
            if (!(delta > 0.0) || !isfinite(delta)) {
                brk = 1;
                break;
            }
            const double alpha = gam / delta;
            const double a = alpha;
            for (int i = tid; i < g.ns; i += bs) w.x[i] = fma(a, w.p[i], w.x[i]);
            for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {
                const int tile = t >> 4, q = t & 15;
                const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
                const int pp = (ty * TILE + (q >> 2) + g.hk) * g.Wp + tx * TILE + (q & 3) + g.xoff;
                w.rimg[pp] = fma(-a, w.qimg[pp], w.rimg[pp]);
            }
            __syncthreads();
            if (twin) {
                apply_A(ph);
                for (int i = tid; i < g.ns; i += bs) xh[i] = fma(a, ph[i], xh[i]);
                for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {
                    const int tile = t >> 4, q = t & 15;
                    const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
                    const int pp = (ty * TILE + (q >> 2) + g.hk) * g.Wp + tx * TILE + (q & 3) + g.xoff;
                    rh[pp] = fma(-a, w.qimg[pp], rh[pp]);
                }
                __syncthreads();
            }
            // s = A^T r, beta = ||s||^2 / gamma, p = s + beta p
            const double gnew = block_sum(apply_AT(w.rimg, w.s), red, which);
            which ^= 1;
            const double beta = gnew / gam;
            gam = gnew;
            if (twin) apply_AT(rh, sh);
            const double bt = beta;
            double xx = 0.0;
            for (int i = tid; i < g.ns; i += bs) {
                w.p[i] = fma(bt, w.p[i], w.s[i]);
                if (twin) ph[i] = fma(bt, ph[i], sh[i]);
                xx += w.x[i] * w.x[i];
                iters_x[(size_t)k * pn + i] = w.x[i];
            }
            // records: chi^2_k = ||r_k||^2, sum s_k^2, twin dof_k = bhat^T rhat_k
            double rr = 0.0, br = 0.0;
            for (int t = tid; t < g.ntiles * (TILE * TILE); t += bs) {
                const int tile = t >> 4, q = t & 15;
                const int ty = tile / g.tiles_x, tx = tile - ty * g.tiles_x;
                const int y = ty * TILE + (q >> 2), x = tx * TILE + (q & 3);
                const int pp = (y + g.hk) * g.Wp + x + g.xoff;
                rr += w.rimg[pp] * w.rimg[pp];
                if (twin && x < g.nx && y < g.ny && w.swp[pp] > 0.0) br += (double)bh[y * g.nx + x] * rh[pp];
            }
            rr = block_sum(rr, red, which);
            which ^= 1;
            xx = block_sum(xx, red, which);
            which ^= 1;
            if (twin) {
                br = block_sum(br, red, which);
                which ^= 1;
            }
            if (tid == 0) {
                chi2[k] = rr;
                reg[k] = xx;
                if (dof) dof[k] = twin ? br : 0.0;
            }
            done = k;
        }
        // an early stop repeats the last record (the L-curve merges repeats)
        if (tid == 0)
            for (int k = done + 1; k <= A.n_iter; ++k) {
                chi2[k] = chi2[done];
                reg[k] = reg[done];
                if (dof) dof[k] = dof[done];
            }
        __syncthreads();
        for (int k = done + 1; k <= A.n_iter; ++k)
            for (int i = tid; i < g.ns; i += bs) iters_x[(size_t)k * pn + i] = iters_x[(size_t)done * pn + i];

        // ---- corner of the L-curve over iterations 1..n_iter
        if (tid == 0) {
            int flat = 0, cn = 0;
            if (A.n_iter >= 1) cn = 1 + lcurve_corner_dev(chi2 + 1, reg + 1, A.n_iter, kap, &flat);
            if (A.kappa) {
                A.kappa[(long long)c * n1] = 0.0;
                for (int k = 1; k <= A.n_iter; ++k) A.kappa[(long long)c * n1 + k] = kap[k - 1];
            }
            A.corner[c] = cn;
            A.status[c] = cstat | (flat ? ST_FLAT : 0) | (brk ? ST_BREAK : 0);
            slot[1] = cn;
        }
        __syncthreads();
        if (A.s_out) {
            const int cn = slot[1];
            for (int i = tid; i < A.max_ns; i += bs)
                A.s_out[(long long)c * A.max_ns + i] = i < g.ns ? (T)iters_x[(size_t)cn * pn + i] : (T)0;
        }
    }
}

}  // namespace mirage
