// Host stand-ins for the CUDA names fftconv.cuh uses, for running a CTA's
// code on real host threads: each thread has its own threadIdx, blockDim is
// the thread count, and __syncthreads() is a barrier across them.  Built
// with ThreadSanitizer, any two threads touching the same element between
// barriers (one of them writing) is reported.
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
extern thread_local HostDim threadIdx;
extern HostDim blockDim;
void host_cta_barrier();
#define __device__
#define __host__
#define __forceinline__ inline
#define __syncthreads() host_cta_barrier()
inline void sincospi(double a, double* s, double* c) {
    const double pi = 3.14159265358979323846;
    *s = std::sin(pi * a);
    *c = std::cos(pi * a);
}
using std::fmax;
using std::hypot;
using std::isfinite;
using std::min;
