// The lens model of the ray trace (Eq. thinlens; Eqs. SIEX/SIEY; external
// shear), shared by the ray-trace kernels; host-callable so that the tests
// can run it against the oracle's lens model.
#pragma once

#include <cuda_runtime.h>

namespace mirage {

__host__ __device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__host__ __device__ __forceinline__ double m_atan(double x) { return atan(x); }
__host__ __device__ __forceinline__ float m_atanh(float x) { return atanhf(x); }
__host__ __device__ __forceinline__ double m_atanh(double x) { return atanh(x); }
__host__ __device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__host__ __device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__host__ __device__ __forceinline__ double m_floor(double x) { return floor(x); }

template <typename T>
struct LensT {
    T b, q, c, s, x0, y0, g1, g2, bqf, f;
    int sis, bad;
};

template <typename T>
__host__ __device__ LensT<T> make_lens(const double* l) {
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
__host__ __device__ __forceinline__ void trace_ray(const LensT<T>& L, T tx, T ty, T& bx, T& by) {
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

}  // namespace mirage
