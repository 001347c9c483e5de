// Source-plane interpolation weights shared by the kernels (host-callable
// so that the tests can check them against the oracle's definitions).
#pragma once

#include <cuda_runtime.h>

namespace mirage {

// Bicubic interpolation (Section 2.1 lists it beside bilinear): Keys'
// cubic-convolution kernel with a = -1/2, W(t) = 3/2|t|^3 - 5/2|t|^2 + 1 on
// |t| <= 1 and -1/2|t|^3 + 5/2|t|^2 - 4|t| + 2 on 1 < |t| < 2.  A ray at
// offset u in its cell weighs the centres at -1, 0, 1, 2 along each axis by
// W(1 + u), W(u), W(1 - u), W(2 - u), written out below as cubics in u.
// Centres beyond the grid hold no source and are skipped.
template <typename V>
__host__ __device__ __forceinline__ V keys_weight(int i, V u) {
    const V u2 = u * u, u3 = u2 * u;
    switch (i) {
        case 0: return (V)0.5 * (-u3 + (V)2 * u2 - u);
        case 1: return (V)0.5 * ((V)3 * u3 - (V)5 * u2 + (V)2);
        case 2: return (V)0.5 * ((V)-3 * u3 + (V)4 * u2 + u);
        default: return (V)0.5 * (u3 - u2);
    }
}

}  // namespace mirage
