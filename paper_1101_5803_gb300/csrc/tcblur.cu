// The PSF blur B (Section 2.2) of a batch of images on two engines, to
// measure a tensor-core form of the convolutions of the FP32 CG inner
// solves against the FFMA register tiles those solves use.
//
//  * k_blur_ffma: the CG kernel's own convolution (conv_tile_fast: one 4 x 4
//    output tile per thread, PSF taps as kernel parameters read by FFMA from
//    the constant bank) on a zero-padded image in shared memory.
//  * k_blur_tc: block-Toeplitz products on the tcgen05 tensor cores.  The
//    image is cut into strips of 16 output columns.  Output row y of strip s
//    is, summed over the PSF rows i, the padded input row segment
//    X(y + i, 16 s ... 16 s + 23) times the 24 x 16 Toeplitz matrix
//    T_i[c][n] = f(i, c - n) (zero unless 0 <= c - n < K), f the PSF as a
//    correlation kernel.  The strips' rows are stacked one after another
//    (strip s, padded row r -> row s R + r, R = ny + K - 1), so one MMA takes
//    M = 128 consecutive stacked rows: A is a window of the stacked image
//    (K-major core matrices of 8 rows x 4 values, which is the image stored
//    column-quad-major: no copy per PSF row, only a start-address shift), B
//    is T_i (N = 16), K = 24 per PSF row in three TF32 steps of 8.  A tile's
//    K x 3 products accumulate in one 16-column block of tensor memory;
//    rows whose padded row is past the image are computed and dropped.
//    Operands are rounded to TF32 (nearest) when stored; accumulation is
//    FP32.
// Both engines keep the image in shared memory for `reps` applications in
// a row (the way the inner solves reuse it), so the timing measures the
// convolution, not the image's trip through HBM.  The tensor-core engine
// needs one image buffer (about 38 KB at 64 x 64) beside the Toeplitz
// operands (14 KB): a blur's result overwrites its input once the products
// have completed, and four CTAs share an SM, so that one CTA's products
// overlap the others' stores.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/mirage.h"
#include "fast.cuh"
#include "tc05.cuh"

namespace mirage {
namespace {

thread_local std::string g_blur_err;

int blur_fail(int code, const std::string& msg) {
    g_blur_err = msg;
    return code;
}

// ------------------------------------------------------------ FFMA engine
struct BlurArgs {
    const float* img;
    float* out;
    int n, nx, ny, reps, Wp;
    float tap[MAX_PTAP];  // correlation taps f(i, j), row-major K x K
};

template <int K>
struct FfmaLayout {
    static constexpr int H = (K - 1) / 2;
    static constexpr int XOFF = xoff_of<float>(H);                     // image column 0 in the buffer
    static constexpr int NVW = (TILE + K - 1 + XOFF - H + 3) / 4 * 4;  // columns one tile row reads
    __host__ __device__ static int wp(int nx) {
        const int a = (nx - TILE + NVW + 3) / 4 * 4, b = (XOFF + nx + H + 3) / 4 * 4;
        return a > b ? a : b;
    }
    // rows: the image rounded up to whole tiles plus the halo, so that the
    // last tile row's reads stay inside its buffer
    __host__ __device__ static int rows(int ny) { return (ny + TILE - 1) / TILE * TILE + 2 * H; }
    static size_t smem(int nx, int ny) { return 2 * sizeof(float) * (size_t)rows(ny) * wp(nx); }
};

template <int K>
__global__ void __launch_bounds__(NTHREADS) k_blur_ffma(const __grid_constant__ BlurArgs A) {
    using Lay = FfmaLayout<K>;
    constexpr int H = Lay::H;
    extern __shared__ __align__(16) float fb[];
    const int Wp = A.Wp, rows = Lay::rows(A.ny), tx_n = A.nx / TILE, ntile = tx_n * ((A.ny + TILE - 1) / TILE);
    float* buf[2] = {fb, fb + rows * Wp};
    for (int e = threadIdx.x; e < 2 * rows * Wp; e += blockDim.x) fb[e] = 0.f;
    __syncthreads();
    for (int img = blockIdx.x; img < A.n; img += gridDim.x) {
        const float* src = A.img + (size_t)img * A.nx * A.ny;
        float* dst = A.out + (size_t)img * A.nx * A.ny;
        for (int e = threadIdx.x; e < A.nx * A.ny; e += blockDim.x) {
            const int y = e / A.nx, x = e - y * A.nx;
            buf[0][(y + H) * Wp + x + Lay::XOFF] = src[e];
        }
        __syncthreads();
        for (int rep = 0; rep < A.reps; ++rep) {
            const float* cur = buf[rep & 1];
            float* nxt = buf[(rep + 1) & 1];
            const bool last = rep == A.reps - 1;
            for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
                const int ty = t / tx_n, tx = t - ty * tx_n;
                float o16[16];
                conv_tile_fast<K, TAPS_PARAM>(cur + ty * TILE * Wp + tx * TILE, Wp, nullptr, A.tap, o16);
#pragma unroll
                for (int r = 0; r < TILE; ++r) {
                    const int y = ty * TILE + r;
                    if (y >= A.ny) break;
                    const float4 v = make_float4(o16[r * 4], o16[r * 4 + 1], o16[r * 4 + 2], o16[r * 4 + 3]);
                    if (last)
                        *reinterpret_cast<float4*>(dst + (size_t)y * A.nx + tx * TILE) = v;
                    else
                        *reinterpret_cast<float4*>(nxt + (y + H) * Wp + tx * TILE + Lay::XOFF) = v;
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------ tensor-core engine
constexpr int TC_STRIP = 16;  // output columns per strip (the MMA's N)
constexpr int TC_M = 128;     // stacked rows per MMA

template <int K>
struct TcLayout {
    static constexpr int H = (K - 1) / 2;
    static constexpr int WIN = (TC_STRIP + K - 1 + 7) / 8 * 8;  // window columns per strip (K steps of 8)
    static constexpr int CG = WIN / 4;                          // column quads per window
    static constexpr int KS = WIN / 8;                          // MMA K steps per PSF row
    static constexpr size_t toeplitz_bytes = (size_t)K * CG * 2 * 128;
    int S, R, T, F, tcols;
    TcLayout(int nx, int ny) {
        S = nx / TC_STRIP;
        R = ny + 2 * H;
        T = (S * R + TC_M - 1) / TC_M;
        F = T * TC_M + 8;  // stacked rows held (the last tile's rows plus the PSF-row shifts)
        tcols = 32;
        while (tcols < TC_STRIP * T) tcols *= 2;
    }
    size_t buf_bytes() const { return (size_t)CG * F * 16; }
    size_t smem() const { return toeplitz_bytes + buf_bytes() + 16; }
};

struct TcArgs {
    const float* img;
    float* out;
    int n, nx, ny, reps;
    int S, R, T, F, tcols;
    float tap[MAX_PTAP];
};

// one quad of 4 consecutive image values (row y, columns 16 s + 4 q ...) into
// every strip window that holds it: strip s2's window position
// c = 4 q + H + 16 (s - s2), column quad c / 4, stacked row s2 R + y + H
template <int K>
__device__ __forceinline__ void tc_put_quad(float* buf, const TcArgs& A, int s, int y, int q, float4 v) {
    using Lay = TcLayout<K>;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        const int s2 = s + d;
        const int c = 4 * q + Lay::H - TC_STRIP * d;
        if (s2 < 0 || s2 >= A.S || c < 0 || c >= Lay::WIN) continue;
        reinterpret_cast<float4*>(buf)[(c >> 2) * A.F + s2 * A.R + y + Lay::H] = v;
    }
}

__device__ __forceinline__ float4 tf32_4(float4 v) {
    return make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
}

template <int K>
__global__ void __launch_bounds__(128) k_blur_tc(const __grid_constant__ TcArgs A) {
    using namespace tc05;
    using Lay = TcLayout<K>;
    static_assert(Lay::H % 4 == 0, "image quads must map onto window quads");
    constexpr uint32_t ID = idesc(FMT_TF32, TC_M, TC_STRIP);
    extern __shared__ __align__(128) unsigned char tb[];
    float* sT = reinterpret_cast<float*>(tb);
    float* X = reinterpret_cast<float*>(tb + Lay::toeplitz_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(X + (size_t)Lay::CG * A.F * 4);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(slot, (uint32_t)A.tcols);
    if (threadIdx.x == 0) bar_init(bar, 1);
    // Toeplitz operands, K-major: PSF row i, column quad kc, row group g
    // (n = 8 g + r), element e -> byte ((i CG + kc) 2 + g) 128 + 16 r + 4 e
    for (int e = threadIdx.x; e < K * Lay::CG * 2 * 32; e += blockDim.x) {
        const int el = e & 3, r = (e >> 2) & 7, g = (e >> 5) & 1, rest = e >> 6;
        const int kc = rest % Lay::CG, i = rest / Lay::CG;
        const int n = 8 * g + r, c = 4 * kc + el, j = c - n;
        sT[e] = (j >= 0 && j < K) ? tf32_round(A.tap[i * K + j]) : 0.f;
    }
    for (size_t e = threadIdx.x; e < (size_t)Lay::CG * A.F * 4; e += blockDim.x) X[e] = 0.f;
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t aT = saddr(sT), aX = saddr(X);
    const uint32_t lbo_a = (uint32_t)A.F * 16u;
    const int q_per_row = A.nx / 4;
    uint32_t phase = 0;
    bool ok = true;
    for (int img = blockIdx.x; img < A.n; img += gridDim.x) {
        const float* src = A.img + (size_t)img * A.nx * A.ny;
        float* dst = A.out + (size_t)img * A.nx * A.ny;
        if (ok) {
            for (int e = threadIdx.x; e < A.ny * q_per_row; e += blockDim.x) {
                const int y = e / q_per_row, qq = e - y * q_per_row;
                const float4 v = reinterpret_cast<const float4*>(src)[e];
                tc_put_quad<K>(X, A, qq >> 2, y, qq & 3, tf32_4(v));
            }
        }
        for (int rep = 0; rep < A.reps && ok; ++rep) {
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            if (threadIdx.x == 0) {
                fence_after_sync();
                for (int t = 0; t < A.T; ++t)
                    for (int i = 0; i < K; ++i)
#pragma unroll
                        for (int ks = 0; ks < Lay::KS; ++ks) {
                            const uint64_t da =
                                sdesc(aX + (uint32_t)((2 * ks) * A.F + TC_M * t + i) * 16u, lbo_a, 128);
                            const uint64_t db = sdesc(aT + (uint32_t)((i * Lay::CG + 2 * ks) * 2) * 128u, 256, 128);
                            mma_tf32(tmem + (uint32_t)(TC_STRIP * t), da, db, ID, (i > 0 || ks > 0) ? 1u : 0u);
                        }
                commit(bar);
            }
            ok = __syncthreads_and(bar_wait(bar, phase)) != 0;  // one decision for the whole CTA
            phase ^= 1;
            fence_after_sync();
            if (!ok) break;
            const bool last = rep == A.reps - 1;
            for (int t = 0; t < A.T; ++t) {
                float v[16];
                ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(TC_STRIP * t), v);
                const int f = TC_M * t + warp * 32 + lane;
                const int s = f / A.R, y = f - s * A.R;
                if (s >= A.S || y >= A.ny) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    if (last)
                        reinterpret_cast<float4*>(dst + (size_t)y * A.nx)[s * 4 + q] = o;
                    else
                        tc_put_quad<K>(X, A, s, y, q, tf32_4(o));
                }
            }
        }
        if (!ok) {  // a completion wait ran out: this image and the rest are NaN
            for (int e = threadIdx.x; e < A.nx * A.ny; e += blockDim.x) dst[e] = __int_as_float(0x7fc00000);
        }
    }
    if (!ok) bar_wait(bar, phase ^ 1);  // (bounded) for the products still in flight
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, (uint32_t)A.tcols);
}

}  // namespace
}  // namespace mirage

extern "C" {

int mirage_psf_blur(int engine, const float* img, float* out, int n, int nx, int ny, const float* psf, int K,
                    int reps, void* stream) {
    using namespace mirage;
    if (engine != MIRAGE_BLUR_FFMA && engine != MIRAGE_BLUR_TC_TF32)
        return blur_fail(MIRAGE_ERR_ARG, "psf_blur: unknown engine");
    if (K != 9) return blur_fail(MIRAGE_ERR_UNSUPPORTED, "psf_blur: K must be 9");
    if (n < 0 || reps < 1 || nx < 16 || nx % 16 != 0 || ny < 1 || ny > 4096)
        return blur_fail(MIRAGE_ERR_ARG, "psf_blur: bad sizes (nx a positive multiple of 16, ny >= 1, reps >= 1)");
    if (!psf || (n > 0 && (!img || !out)) || ((uintptr_t)img | (uintptr_t)out) % 16 != 0)
        return blur_fail(MIRAGE_ERR_ARG, "psf_blur: null or unaligned pointer (16 bytes)");
    if (n == 0) return MIRAGE_OK;
    int dev = 0, smem_max = 0, smem_sm = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return blur_fail(MIRAGE_ERR_CUDA, "psf_blur: device query failed");
    cudaStream_t st = (cudaStream_t)stream;
    // correlation taps: B x (y, x) = sum psf(i, j) x(y - i + h, x - j + h)
    //                              = sum f(i, j) x(y + i - h, x + j - h), f = psf flipped
    float tap[MAX_PTAP];
    for (int i = 0; i < K * K; ++i) tap[i] = psf[K * K - 1 - i];
    // resident CTAs per SM follow from the shared memory each takes (1 KB of
    // it reserved per CTA); the grid is that many per SM, or one per image
    if (engine == MIRAGE_BLUR_FFMA) {
        using Lay = FfmaLayout<9>;
        const size_t smem = Lay::smem(nx, ny);
        if (smem > (size_t)smem_max) return blur_fail(MIRAGE_ERR_UNSUPPORTED, "psf_blur: image too large");
        BlurArgs A{};
        A.img = img;
        A.out = out;
        A.n = n;
        A.nx = nx;
        A.ny = ny;
        A.reps = reps;
        A.Wp = Lay::wp(nx);
        std::copy(tap, tap + K * K, A.tap);
        if (cudaFuncSetAttribute(k_blur_ffma<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return blur_fail(MIRAGE_ERR_CUDA, "psf_blur: shared-memory attribute");
        const int per_sm = std::max(1, std::min(smem_sm / (int)(smem + 1024), 2048 / NTHREADS));
        k_blur_ffma<9><<<std::min(n, sms * per_sm), NTHREADS, smem, st>>>(A);
    } else {
        using Lay = TcLayout<9>;
        const Lay L(nx, ny);
        if (L.smem() > (size_t)smem_max || L.tcols > 512)
            return blur_fail(MIRAGE_ERR_UNSUPPORTED, "psf_blur: image too large for the tensor-core engine");
        TcArgs A{};
        A.img = img;
        A.out = out;
        A.n = n;
        A.nx = nx;
        A.ny = ny;
        A.reps = reps;
        A.S = L.S;
        A.R = L.R;
        A.T = L.T;
        A.F = L.F;
        A.tcols = L.tcols;
        std::copy(tap, tap + K * K, A.tap);
        if (cudaFuncSetAttribute(k_blur_tc<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem()) !=
            cudaSuccess)
            return blur_fail(MIRAGE_ERR_CUDA, "psf_blur: shared-memory attribute");
        // (tensor memory: every resident CTA holds tcols of the SM's 512 columns)
        const int per_sm = std::max(1, std::min(smem_sm / (int)(L.smem() + 1024), 512 / L.tcols));
        k_blur_tc<9><<<std::min(n, sms * per_sm), 128, L.smem(), st>>>(A);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return blur_fail(MIRAGE_ERR_CUDA, std::string("psf_blur: ") + cudaGetErrorString(e));
    return MIRAGE_OK;
}

const char* mirage_blur_last_error(void) { return mirage::g_blur_err.c_str(); }

}  // extern "C"
