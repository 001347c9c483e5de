// The solver loops' geometry and the regulariser H of Eq. TKReg (identity,
// forward-difference gradient, 5-point Laplacian; zero beyond the grid),
// host-callable so that the tests can check H, H^T and diag(H^T H) against
// the oracle's explicit matrices.
#pragma once

#include <cuda_runtime.h>

namespace mirage {

// geometry needed inside the solver loops (passed by value)
template <typename T>
struct Geo {
    int nx, ny, sx, sy, ns, nreg, K, hk, kp, xoff, sh, Np, ncx, ncells, Wp, plen, tiles_x, ntiles, reg, nent, interp;
    T invNp;
};

// row `row` of H v (rows ns..2ns-1 are Dy for the gradient); zero beyond the grid
template <typename T, typename V>
__host__ __device__ __forceinline__ V apply_H_row(const Geo<T>& g, const V* __restrict__ v, int row) {
    if (g.reg == 0) return v[row];
    if (g.reg == 2) {
        const int ib = row / g.sx, ia = row - ib * g.sx;
        V acc = (V)4 * v[row];
        if (ia > 0) acc -= v[row - 1];
        if (ia < g.sx - 1) acc -= v[row + 1];
        if (ib > 0) acc -= v[row - g.sx];
        if (ib < g.sy - 1) acc -= v[row + g.sx];
        return acc;
    }
    if (row < g.ns) {
        const int ib = row / g.sx, ia = row - ib * g.sx;
        (void)ib;
        return (ia < g.sx - 1 ? v[row + 1] : (V)0) - v[row];
    }
    const int i = row - g.ns;
    const int ib = i / g.sx;
    return (ib < g.sy - 1 ? v[i + g.sx] : (V)0) - v[i];
}

// (H^T r)_i
template <typename T, typename V>
__host__ __device__ __forceinline__ V apply_HT_at(const Geo<T>& g, const V* __restrict__ r, int i, int ia, int ib) {
    if (g.reg == 0) return r[i];
    if (g.reg == 2) {
        V acc = (V)4 * r[i];
        if (ia > 0) acc -= r[i - 1];
        if (ia < g.sx - 1) acc -= r[i + 1];
        if (ib > 0) acc -= r[i - g.sx];
        if (ib < g.sy - 1) acc -= r[i + g.sx];
        return acc;
    }
    const V* ry = r + g.ns;
    V acc = -r[i] - ry[i];
    if (ia > 0) acc += r[i - 1];
    if (ib > 0) acc += ry[i - g.sx];
    return acc;
}

// diag(H^T H) at source pixel (ia, ib): identity 1; gradient 2 + [left
// neighbour] + [lower neighbour]; Laplacian 16 + number of neighbours
template <typename T>
__host__ __device__ __forceinline__ T hth_diag_at(const Geo<T>& g, int ia, int ib) {
    if (g.reg == 0) return (T)1;
    if (g.reg == 1) return (T)(2 + (ia > 0) + (ib > 0));
    return (T)(16 + (ia > 0) + (ia < g.sx - 1) + (ib > 0) + (ib < g.sy - 1));
}

}  // namespace mirage
