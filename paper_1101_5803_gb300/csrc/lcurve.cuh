// L-curve corner of one candidate (Section 2.6), shared by the finalize and
// L-curve kernels; host-callable so that the tests can run it against the
// oracle's spline corner on many curves.
//
// Points (log10 R_k, log10 chi2_k) in lambda order, parametrised by their
// cumulative chord length; points closer than 1e-12 of the total length to
// their predecessor are merged; natural cubic splines through the kept
// points (second derivatives by the Thomas algorithm); the corner is the
// knot of largest curvature |x' y'' - y' x''| / (x'^2 + y'^2)^(3/2).
// Fewer than three kept points, or a curvature times the total length below
// 1e-9 everywhere, is flat: the middle index with *flat = 1.
#pragma once

#include <cuda_runtime.h>

namespace mirage {

constexpr int MAX_LAM = 64;  // longest lambda grid of one candidate

__host__ __device__ inline int lcurve_corner_dev(const double* chi2, const double* reg, int n, double* kappa,
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

}  // namespace mirage
