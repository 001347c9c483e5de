// FFT convolution with the PSF, one CTA per image (Section 2.2: the paper
// applies B through the Fourier transform).  Used for PSFs too wide for the
// direct K x K tile convolution to pay.
//
// B x = crop(IFFT2(FFT2(x) * S)) on an M x M grid, M a power of two with
// M >= max(nx, ny) + (K - 1) / 2, S the transform of the PSF placed with its
// centre at index (0, 0) (wrapped), divided by M^2.  The wrap of that
// centred placement lands only in the zero padding, so the crop equals the
// zero-padded linear convolution; B^T (the correlation) uses conj(S).
//
// Layout: half spectra (kx = 0 .. M/2, the input is real) stored kx-major,
// F[kx * M + ky], so that the column transforms read contiguous memory.
// Rows are transformed two at a time (one real row in the real part, the
// next in the imaginary part, separated after the transform by the
// Hermitian symmetry of real input).  The transforms themselves are
// radix-4 Stockham (self-sorting) passes, with one radix-2 pass for odd
// log2 M, over a batch of rows held in shared memory, with per-stage
// twiddle tables.
#pragma once

#include <cuda_runtime.h>

namespace mirage {

template <typename R>
struct CxOf;
template <>
struct CxOf<float> {
    using type = float2;
};
template <>
struct CxOf<double> {
    using type = double2;
};

constexpr int FFT_BUF_BYTES = 64 * 1024;  // shared ping-pong buffers of one batch

template <typename R>
struct FftPlan {
    using C = typename CxOf<R>::type;
    int M = 0, logM = 0, nb = 0;  // size, log2(size), transforms per batch
    const C* tw = nullptr;        // shared [M - 1]: stage ns uses tw[ns - 1 + k] = exp(-i pi k / ns), k < ns
    C* b0 = nullptr;              // shared [nb][M + 1] (row stride M + 1 against bank conflicts)
    C* b1 = nullptr;
    C* F = nullptr;        // global work [(M/2 + 1) * M], kx-major
    const C* S = nullptr;  // global spectrum [(M/2 + 1) * M], kx-major, scaled by 1 / M^2
};

// smallest power of two >= n (n >= 1)
__host__ __device__ inline int fft_size_for(int n) {
    int m = 1;
    while (m < n) m <<= 1;
    return m;
}

// shared bytes of the FFT path for size M: two plans, both twiddle tables
// (with alignment slack) and the batch buffers
__host__ __device__ inline size_t fft_smem_bytes(int M) {
    return 128 + (size_t)(M - 1) * (sizeof(float2) + sizeof(double2)) + 64 + FFT_BUF_BYTES;
}

// transforms per batch for element type C
template <typename C>
__host__ __device__ inline int fft_batch_count(int M) {
    const int nb = FFT_BUF_BYTES / (int)(2 * (M + 1) * sizeof(C));
    return nb < 1 ? 1 : nb;
}

template <typename C>
__device__ __forceinline__ C cx(decltype(C::x) re, decltype(C::x) im) {
    C z;
    z.x = re;
    z.y = im;
    return z;
}

// per-stage twiddles: tw[ns - 1 + k] = exp(-i pi k / ns) for ns = 1, 2, ..., M/2
template <typename R>
__device__ void fft_twiddles(typename CxOf<R>::type* tw, int M) {
    using C = typename CxOf<R>::type;
    for (int i = threadIdx.x; i < M - 1; i += blockDim.x) {
        int ns = 1;
        while (2 * ns - 1 <= i) ns <<= 1;
        const int k = i - (ns - 1);
        double s, c;
        sincospi(-(double)k / (double)ns, &s, &c);
        tw[i] = cx<C>((R)c, (R)s);
    }
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return cx<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// nb transforms of length M, transform f at x + f * (M + 1); Stockham
// (self-sorting) passes ping-ponging between x and y: radix 4 while two
// factors of two remain, then one radix-2 pass for odd log2 M.  A radix-r
// pass at span ns takes, for j < M / r and k = j mod ns, the inputs
// x[j + q M / r] (q < r) times exp(-+2 pi i q k / (r ns)), their length-r
// DFT, and writes output p to (j - k) r + k + p ns.  Every thread of the
// CTA takes part; the data must be complete (barrier) before the call.
// Returns the buffer that holds the result.
template <typename R>
__device__ typename CxOf<R>::type* fft_batch(typename CxOf<R>::type* x, typename CxOf<R>::type* y,
                                             const typename CxOf<R>::type* tw, int M, int logM, int nb, bool inverse) {
    using C = typename CxOf<R>::type;
    const int ld = M + 1;
    int ns = 1, lg = logM;
    for (; lg >= 2; lg -= 2, ns <<= 2) {
        const int q = M >> 2, lq = logM - 2;
        for (int t = threadIdx.x; t < (nb << lq); t += blockDim.x) {
            const int f = t >> lq, j = t & (q - 1);
            const C* xf = x + f * ld;
            C* yf = y + f * ld;
            const int k = j & (ns - 1);
            C w1 = tw[2 * ns - 1 + k];  // exp(-i pi k / (2 ns)) = exp(-2 pi i k / (4 ns))
            if (inverse) w1.y = -w1.y;
            const C w2 = cmul(w1, w1), w3 = cmul(w2, w1);
            const C a = xf[j], b = cmul(w1, xf[j + q]), c = cmul(w2, xf[j + 2 * q]), d = cmul(w3, xf[j + 3 * q]);
            const C s0 = cx<C>(a.x + c.x, a.y + c.y), s1 = cx<C>(a.x - c.x, a.y - c.y);
            const C s2 = cx<C>(b.x + d.x, b.y + d.y), s3 = cx<C>(b.x - d.x, b.y - d.y);
            // -i s3 for the forward transform, +i s3 for the inverse
            const C is3 = inverse ? cx<C>(-s3.y, s3.x) : cx<C>(s3.y, -s3.x);
            const int o = ((j - k) << 2) + k;
            yf[o] = cx<C>(s0.x + s2.x, s0.y + s2.y);
            yf[o + ns] = cx<C>(s1.x + is3.x, s1.y + is3.y);
            yf[o + 2 * ns] = cx<C>(s0.x - s2.x, s0.y - s2.y);
            yf[o + 3 * ns] = cx<C>(s1.x - is3.x, s1.y - is3.y);
        }
        __syncthreads();
        C* t = x;
        x = y;
        y = t;
    }
    if (lg == 1) {
        const int half = M >> 1;
        const int nbf = nb << (logM - 1);
        for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
            const int f = t >> (logM - 1), j = t & (half - 1);
            const C* xf = x + f * ld;
            C* yf = y + f * ld;
            const int k = j & (ns - 1);
            C w = tw[ns - 1 + k];
            if (inverse) w.y = -w.y;
            const C a = xf[j], b = cmul(w, xf[j + half]);
            const int o = ((j - k) << 1) + k;
            yf[o] = cx<C>(a.x + b.x, a.y + b.y);
            yf[o + ns] = cx<C>(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
        C* t = x;
        x = y;
        y = t;
    }
    return x;
}

// Row pass: the real rows 0 .. rows_in-1 given by load(y, n) (n < M; the
// loader returns 0 outside its data) into the half spectra F[kx][y].
template <typename R, class Load>
__device__ void fft_rows_forward(const FftPlan<R>& f, Load load, int rows_in) {
    using C = typename CxOf<R>::type;
    const int M = f.M, ld = M + 1, H1 = (M >> 1) + 1;
    for (int y0 = 0; y0 < rows_in; y0 += 2 * f.nb) {
        const int np = min(f.nb, (rows_in - y0 + 1) >> 1);
        for (int t = threadIdx.x; t < (np << f.logM); t += blockDim.x) {
            const int p = t >> f.logM, n = t & (M - 1);
            const int y = y0 + 2 * p;
            const R a = load(y, n);
            const R b = y + 1 < rows_in ? load(y + 1, n) : (R)0;
            f.b0[p * ld + n] = cx<C>(a, b);
        }
        __syncthreads();
        const C* X = fft_batch<R>(f.b0, f.b1, f.tw, M, f.logM, np, false);
        // separate the pair: A_k = (Z_k + conj Z_{-k}) / 2, B_k = (Z_k - conj Z_{-k}) / 2i
        for (int t = threadIdx.x; t < np * H1; t += blockDim.x) {
            const int k = t / np, p = t - k * np;
            const C* Xp = X + p * ld;
            const C z = Xp[k], zm = Xp[(M - k) & (M - 1)];
            const int y = y0 + 2 * p;
            f.F[k * M + y] = cx<C>((R)0.5 * (z.x + zm.x), (R)0.5 * (z.y - zm.y));
            if (y + 1 < rows_in) f.F[k * M + y + 1] = cx<C>((R)0.5 * (z.y + zm.y), (R)0.5 * (zm.x - z.x));
        }
        __syncthreads();
    }
}

// Column pass of a convolution: for every kx, transform F[kx][0 .. rows_in)
// (zero beyond), multiply by S (conj S for the correlation), transform back
// and keep rows 0 .. rows_out-1 in F.
template <typename R>
__device__ void fft_cols_convolve(const FftPlan<R>& f, int rows_in, int rows_out, bool corr) {
    using C = typename CxOf<R>::type;
    const int M = f.M, ld = M + 1, H1 = (M >> 1) + 1;
    for (int k0 = 0; k0 < H1; k0 += f.nb) {
        const int nc = min(f.nb, H1 - k0);
        for (int t = threadIdx.x; t < (nc << f.logM); t += blockDim.x) {
            const int c = t >> f.logM, n = t & (M - 1);
            f.b0[c * ld + n] = n < rows_in ? f.F[(k0 + c) * M + n] : cx<C>((R)0, (R)0);
        }
        __syncthreads();
        C* X = fft_batch<R>(f.b0, f.b1, f.tw, M, f.logM, nc, false);
        C* Y = X == f.b0 ? f.b1 : f.b0;
        for (int t = threadIdx.x; t < (nc << f.logM); t += blockDim.x) {
            const int c = t >> f.logM, n = t & (M - 1);
            C s = f.S[(k0 + c) * M + n];
            if (corr) s.y = -s.y;
            const C z = X[c * ld + n];
            X[c * ld + n] = cx<C>(z.x * s.x - z.y * s.y, z.x * s.y + z.y * s.x);
        }
        __syncthreads();
        const C* Z = fft_batch<R>(X, Y, f.tw, M, f.logM, nc, true);
        for (int t = threadIdx.x; t < nc * rows_out; t += blockDim.x) {
            const int c = t / rows_out, n = t - c * rows_out;
            f.F[(k0 + c) * M + n] = Z[c * ld + n];
        }
        __syncthreads();
    }
}

// Inverse row pass: real rows 0 .. rows_out-1 from the half spectra in F,
// handed to store(y, n, value) for n < cols_out.
template <typename R, class Store>
__device__ void fft_rows_inverse(const FftPlan<R>& f, Store store, int rows_out, int cols_out) {
    using C = typename CxOf<R>::type;
    const int M = f.M, ld = M + 1, half = M >> 1;
    for (int y0 = 0; y0 < rows_out; y0 += 2 * f.nb) {
        const int np = min(f.nb, (rows_out - y0 + 1) >> 1);
        // Z_k = G1_k + i G2_k over the full spectrum, G_{M-k} = conj G_k
        for (int t = threadIdx.x; t < (np << f.logM); t += blockDim.x) {
            const int k = t / np, p = t - k * np;
            const int y = y0 + 2 * p;
            const int kk = k <= half ? k : M - k;
            C g1 = f.F[kk * M + y];
            C g2 = y + 1 < rows_out ? f.F[kk * M + y + 1] : cx<C>((R)0, (R)0);
            if (k > half) {
                g1.y = -g1.y;
                g2.y = -g2.y;
            }
            f.b0[p * ld + k] = cx<C>(g1.x - g2.y, g1.y + g2.x);
        }
        __syncthreads();
        const C* Z = fft_batch<R>(f.b0, f.b1, f.tw, M, f.logM, np, true);
        for (int t = threadIdx.x; t < np * cols_out; t += blockDim.x) {
            const int p = t / cols_out, n = t - p * cols_out;
            const int y = y0 + 2 * p;
            const C z = Z[p * ld + n];
            store(y, n, z.x);
            if (y + 1 < rows_out) store(y + 1, n, z.y);
        }
        __syncthreads();
    }
}

// out = B x (corr = false) or B^T x (corr = true) for real images: rows_in
// rows of input from load, rows_out x cols_out of output to store.
template <typename R, class Load, class Store>
__device__ void fft_convolve(const FftPlan<R>& f, Load load, int rows_in, Store store, int rows_out, int cols_out,
                             bool corr) {
    fft_rows_forward<R>(f, load, rows_in);
    fft_cols_convolve<R>(f, rows_in, rows_out, corr);
    fft_rows_inverse<R>(f, store, rows_out, cols_out);
}

// Spectrum of a K x K PSF centred at (0, 0) on the M x M grid, scaled by
// 1 / M^2, into f.F (kx-major); f.S is not used.
template <typename R, typename P>
__device__ void fft_psf_spectrum(const FftPlan<R>& f, const P* __restrict__ psf, int K) {
    using C = typename CxOf<R>::type;
    const int M = f.M, ld = M + 1, H1 = (M >> 1) + 1, c = (K - 1) >> 1;
    // wrapped placement: tap (a, b) at ((a - c) mod M, (b - c) mod M); when
    // K > M several taps share a grid point (their sum)
    auto load = [&](int y, int n) -> R {
        R v = 0;
        for (int a = (y + c) % M; a < K; a += M)
            for (int b = (n + c) % M; b < K; b += M) v += (R)psf[a * K + b];
        return v;
    };
    fft_rows_forward<R>(f, load, M);
    const R scale = (R)1 / ((R)M * (R)M);
    for (int k0 = 0; k0 < H1; k0 += f.nb) {
        const int nc = min(f.nb, H1 - k0);
        for (int t = threadIdx.x; t < (nc << f.logM); t += blockDim.x) {
            const int cc = t >> f.logM, n = t & (M - 1);
            f.b0[cc * ld + n] = f.F[(k0 + cc) * M + n];
        }
        __syncthreads();
        const C* X = fft_batch<R>(f.b0, f.b1, f.tw, M, f.logM, nc, false);
        for (int t = threadIdx.x; t < (nc << f.logM); t += blockDim.x) {
            const int cc = t >> f.logM, n = t & (M - 1);
            const C z = X[cc * ld + n];
            f.F[(k0 + cc) * M + n] = cx<C>(z.x * scale, z.y * scale);
        }
        __syncthreads();
    }
}

}  // namespace mirage
