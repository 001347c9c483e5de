// Host stand-ins for the few CUDA names fftconv.cuh uses, so that the FFT
// convolution can be compiled with a host compiler and run as one thread:
// the CTA-wide loops then cover every index and the barriers are no-ops
// (work between barriers is independent across threads by construction).
#pragma once
#include <algorithm>
#include <cmath>

struct float2 {
    float x, y;
};
struct double2 {
    double x, y;
};
struct HostDim {
    unsigned x;
};
static const HostDim threadIdx{0}, blockDim{1};
#define __device__
#define __host__
#define __forceinline__ inline
#define __syncthreads() ((void)0)
inline void sincospi(double a, double* s, double* c) {
    const double pi = 3.14159265358979323846;
    *s = std::sin(pi * a);
    *c = std::cos(pi * a);
}
using std::fmax;
using std::hypot;
using std::isfinite;
using std::min;
