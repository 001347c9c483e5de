// Surrogate network: a multilayer perceptron with SiLU hidden layers and a
// linear output layer, trained with mean-squared error and Adam.  Matrix
// products run on the BF16 tcgen05 tensor cores (FP32 accumulate in tensor
// memory);
// master weights, Adam moments, bias, activation and loss stay in FP32.
//
// It predicts, from the encoded lens vector, the standardised
// (log chi2, log10 lambda) of the L-curve corner, so that a genetic
// algorithm can screen its offspring and warm-start the exact solves.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mirage.h"
#include "tc05.cuh"

namespace {

thread_local std::string g_mlp_err;

int mlp_fail(int code, const std::string& msg) {
    g_mlp_err = msg;
    return code;
}

#define MCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return mlp_fail(MIRAGE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// C[M x N] (FP32, row-major, ldc) = sum_k A(m, k) B(k, n) with
//   A(m, k) = A[m * sam + k * sak],  B(k, n) = B[k * sbk + n * sbn]  (BF16)
// on the fifth-generation tensor cores: one CTA of four warps per 128 x BN
// output tile, accumulator in tensor memory (BN FP32 columns), K in chunks
// of TC_BK staged by the CTA into shared memory as K-major core matrices
// (8 rows x 8 BF16), TC_BK / 16 tcgen05.mma of K = 16 per chunk issued by one
// thread, completion through an mbarrier.  Edges are zero-filled.  Should a
// completion wait run out (about a second), the tile is written as NaN.
constexpr int TC_BM = 128, TC_BK = 64;

template <int BN>
constexpr int tc_smem_bytes() {
    return (TC_BM + BN) * TC_BK * 2 + 16;
}

// element (r, k) of a staged tile -> core matrix (r / 8, k / 8), k-chunks
// innermost: BF16 index ((r / 8) * TC_KO + k / 8) * 64 + (r % 8) * 8 + k % 8, so
// one 16-byte row of a core matrix holds 8 consecutive k of one row r
constexpr int TC_KO = TC_BK / 8;  // k-octets (core-matrix columns) per staged row group
__device__ __forceinline__ int tc_at(int r, int k) { return ((r >> 3) * TC_KO + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// How an operand view is staged: rows contiguous along k (16-byte rows of
// 8 k), a transposed view (8 rows contiguous at one k), or element by element
enum : int { ST_KROW = 0, ST_KCOL = 1, ST_SCALAR = 2 };

__device__ __forceinline__ int stage_mode(const __nv_bfloat16* src, long s_row, long s_k) {
    const bool al = ((uintptr_t)src & 15) == 0;
    if (s_k == 1 && (s_row & 7) == 0 && al) return ST_KROW;
    if (s_row == 1 && (s_k & 7) == 0 && al) return ST_KCOL;
    return ST_SCALAR;
}

// One K chunk of a ROWS x TC_BK operand tile: the loads into registers (NV
// 16-byte vectors a thread, all issued before any is used, so their
// latencies overlap one another and the previous chunk's products) ...
template <int ROWS>
struct TcStage {
    static constexpr int NV = ROWS * (TC_BK / 8) / 128;
    uint4 v[NV];

    __device__ __forceinline__ void load(int mode, const __nv_bfloat16* __restrict__ src, long s_row, long s_k,
                                         int r0, int R, int k0, int K) {
        const __nv_bfloat16 z = __float2bfloat16(0.f);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = threadIdx.x + 128 * i;
            v[i] = make_uint4(0u, 0u, 0u, 0u);
            __nv_bfloat16* t = reinterpret_cast<__nv_bfloat16*>(&v[i]);
            if (mode == ST_KROW) {  // row r, k-octet kc
                const int r = e / TC_KO, gr = r0 + r, gk = k0 + 8 * (e % TC_KO);
                if (gr < R && gk + 8 <= K)
                    v[i] = *reinterpret_cast<const uint4*>(src + (long)gr * s_row + gk);
                else if (gr < R)
                    for (int j = 0; j < 8; ++j) t[j] = gk + j < K ? src[(long)gr * s_row + gk + j] : z;
            } else if (mode == ST_KCOL) {  // rows 8 g .. 8 g + 7 at one k
                const int g = e / TC_BK, gr = r0 + 8 * g, gk = k0 + (e - g * TC_BK);
                if (gk < K && gr + 8 <= R)
                    v[i] = *reinterpret_cast<const uint4*>(src + (long)gk * s_k + gr);
                else if (gk < K)
                    for (int j = 0; j < 8; ++j) t[j] = gr + j < R ? src[(long)gk * s_k + gr + j] : z;
            }
        }
    }

    // ... then the stores into the K-major core-matrix layout (the element
    // by element mode loads and stores here)
    __device__ __forceinline__ void store(int mode, __nv_bfloat16* dst, const __nv_bfloat16* __restrict__ src,
                                          long s_row, long s_k, int r0, int R, int k0, int K) const {
        if (mode == ST_SCALAR) {
            const __nv_bfloat16 z = __float2bfloat16(0.f);
            for (int e = threadIdx.x; e < ROWS * TC_BK; e += 128) {
                const int r = e / TC_BK, k = e - r * TC_BK;
                const int gr = r0 + r, gk = k0 + k;
                dst[tc_at(r, k)] = (gr < R && gk < K) ? src[(long)gr * s_row + (long)gk * s_k] : z;
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int e = threadIdx.x + 128 * i;
            if (mode == ST_KROW) {
                *reinterpret_cast<uint4*>(dst + tc_at(e / TC_KO, 8 * (e % TC_KO))) = v[i];
            } else {
                const int g = e / TC_BK, k = e - g * TC_BK;
                const __nv_bfloat16* t = reinterpret_cast<const __nv_bfloat16*>(&v[i]);
#pragma unroll
                for (int j = 0; j < 8; ++j) dst[tc_at(8 * g + j, k)] = t[j];
            }
        }
    }
};

template <int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(const __nv_bfloat16* __restrict__ A, long sam, long sak,
                                                 const __nv_bfloat16* __restrict__ B, long sbk, long sbn,
                                                 float* __restrict__ C, int ldc, int M, int N, int K) {
    using namespace mirage::tc05;
    constexpr int TCOLS = BN < 32 ? 32 : BN;  // a power of two >= 32
    constexpr uint32_t ID = idesc(FMT_BF16, TC_BM, BN);
    extern __shared__ __align__(128) unsigned char tc_sm[];
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(tc_sm);
    __nv_bfloat16* sB = sA + TC_BM * TC_BK;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + BN * TC_BK);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // B(k, n) is staged as rows n: row stride sbn, k stride sbk
    const int ma = stage_mode(A, sam, sak), mb = stage_mode(B, sbn, sbk);
    TcStage<TC_BM> ra;
    TcStage<BN> rb;
    ra.load(ma, A, sam, sak, m0, M, 0, K);
    rb.load(mb, B, sbn, sbk, n0, N, 0, K);
    if (warp == 0) tmem_alloc(slot, TCOLS);
    if (threadIdx.x == 0) bar_init(bar, 1);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *slot;
    bool ok = true;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K && ok; k0 += TC_BK) {
        ra.store(ma, sA, A, sam, sak, m0, M, k0, K);
        rb.store(mb, sB, B, sbn, sbk, n0, N, k0, K);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after_sync();
#pragma unroll
            for (int s = 0; s < TC_BK / 16; ++s) {
                // K step s: core-matrix columns 2s and 2s + 1 (128 B apart),
                // 8-row groups TC_KO * 128 B apart
                const uint64_t da = sdesc(saddr(sA) + s * 256, 128, TC_KO * 128);
                const uint64_t db = sdesc(saddr(sB) + s * 256, 128, TC_KO * 128);
                mma_bf16(tmem, da, db, ID, (k0 > 0 || s > 0) ? 1u : 0u);
            }
            commit(bar);
        }
        if (k0 + TC_BK < K) {  // the next chunk's loads overlap these products
            ra.load(ma, A, sam, sak, m0, M, k0 + TC_BK, K);
            rb.load(mb, B, sbn, sbk, n0, N, k0 + TC_BK, K);
        }
        ok = __syncthreads_and(bar_wait(bar, phase)) != 0;  // one decision for the whole CTA
        phase ^= 1;
        fence_after_sync();
    }
    if (!ok) bar_wait(bar, phase ^ 1);  // (bounded) for the MMAs still in flight
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (row < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + j;
                if (col < N) C[(long)row * ldc + col] = (ok && K > 0) ? v[j] : (K > 0 ? __int_as_float(0x7fc00000) : 0.f);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, TCOLS);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_g(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// x (FP32) -> BF16 activations; with idx, row j of the batch is row idx[j] of x
__global__ void k_to_bf16(const float* __restrict__ x, const int* __restrict__ idx, int cols,
                          __nv_bfloat16* __restrict__ a, long n) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long src = idx ? (long)idx[i / cols] * cols + i % cols : i;
    a[i] = __float2bfloat16(x[src]);
}

// Z += b (per column); hidden layers: A = bf16(silu(Z)); output layer: Y = Z
__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ b, int n, int cols, int hidden,
                           __nv_bfloat16* __restrict__ Aout, float* __restrict__ Y) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)n * cols) return;
    const float z = Z[i] + b[i % cols];
    Z[i] = z;
    if (hidden)
        Aout[i] = __float2bfloat16(silu_f(z));
    else
        Y[i] = z;
}

// dY = 2 (Y - T) / (n cols); loss partial sums.  With idx, row j of the
// batch targets row idx[j] of T.
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, const int* __restrict__ idx,
                            int cols, long total, float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZh,
                            double* __restrict__ loss) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < total) {
        const long ti = idx ? (long)idx[i / cols] * cols + i % cols : i;
        const float d = Y[i] - T[ti];
        dZ[i] = 2.f * d / (float)total;
        dZh[i] = __float2bfloat16(dZ[i]);
        l = (double)d * (double)d;
    }
    if (loss) {
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / (double)total);
    }
}

// dZ = dA * silu'(Z) (hidden layer), also its BF16 copy
__global__ void k_act_back(const float* __restrict__ dA, const float* __restrict__ Z, long total,
                           float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZh) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float d = dA[i] * silu_g(Z[i]);
    dZ[i] = d;
    dZh[i] = __float2bfloat16(d);
}

// db[j] = sum_m dZ[m][j] (fixed order, one thread per column)
__global__ void k_colsum(const float* __restrict__ dZ, int n, int cols, float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int m = 0; m < n; ++m) s += dZ[(long)m * cols + j];
    db[j] = s;
}

// Adam on every parameter; refresh the BF16 copy of the weights
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ ph, const unsigned char* __restrict__ is_w) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (is_w[i]) ph[i] = __float2bfloat16(w);
}

// Adam whose bias corrections follow the device step counter (steps taken
// so far, before this one), for the device-side training loop
__global__ void k_adam_dev(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, long n, float lr, float b1, float b2, float eps,
                           const long long* __restrict__ dstep, __nv_bfloat16* __restrict__ ph,
                           const unsigned char* __restrict__ is_w) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = (float)(*dstep + 1);
    const float c1 = 1.f - powf(b1, s), c2 = 1.f - powf(b2, s);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (is_w[i]) ph[i] = __float2bfloat16(w);
}

// Minibatch rows of one training step: row slot j draws row
// h(seed, step, j) mod n with h the splitmix64 finaliser (a counter-based
// hash: the draw depends only on its three inputs)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_sample_rows(int* __restrict__ idx, int batch, int n, unsigned long long seed,
                              const long long* __restrict__ dstep) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= batch) return;
    const unsigned long long key =
        seed * 0x9E3779B97F4A7C15ull + ((unsigned long long)*dstep << 24) + (unsigned long long)j;
    idx[j] = (int)(mix64(key) % (unsigned long long)n);
}
__global__ void k_step_inc(long long* dstep) { *dstep += 1; }

__global__ void k_params_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ ph, long n) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) ph[i] = __float2bfloat16(p[i]);
}

struct Buf {
    void* p = nullptr;
    size_t n = 0;
    int ensure(size_t bytes) {
        if (bytes <= n) return MIRAGE_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return mlp_fail(MIRAGE_ERR_NOMEM, "mlp: cudaMalloc failed");
        n = bytes;
        return MIRAGE_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

inline unsigned blocks(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

struct mirage_mlp {
    int device = 0;
    int L = 0;                 // weight layers
    std::vector<int> dims;     // L + 1
    std::vector<long> w_off, b_off;
    long n_params = 0;
    int step = 0;
    float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    Buf P, PH, M, V, G, ISW;   // params FP32, BF16 copy, Adam m, v, grads, weight mask
    Buf Z, A, DZ, DZH, DA, LOSS;  // per-batch work (grown on demand)
    Buf IDX, DSTEP;            // device-side training loop: minibatch rows, step counter
    cudaStream_t cap = nullptr;  // private stream on which the training step is captured
    long cap_rows = 0;
    std::vector<long> z_off, a_off;  // per layer offsets into Z / A (elements)
};

namespace {

int ensure_batch(mirage_mlp* m, int n) {
    if (n <= m->cap_rows) return MIRAGE_OK;
    long zt = 0, at = 0;
    m->z_off.assign(m->L + 1, 0);
    m->a_off.assign(m->L + 1, 0);
    int maxw = 0;
    for (int l = 0; l <= m->L; ++l) {
        m->a_off[l] = at;
        at += (long)n * m->dims[l];
        maxw = std::max(maxw, m->dims[l]);
        if (l > 0) {
            m->z_off[l] = zt;
            zt += (long)n * m->dims[l];
        }
    }
    int r;
    if ((r = m->Z.ensure(sizeof(float) * zt))) return r;
    if ((r = m->A.ensure(sizeof(__nv_bfloat16) * at))) return r;
    if ((r = m->DZ.ensure(sizeof(float) * (long)n * maxw))) return r;
    if ((r = m->DZH.ensure(sizeof(__nv_bfloat16) * (long)n * maxw))) return r;
    if ((r = m->DA.ensure(sizeof(float) * (long)n * maxw))) return r;
    if ((r = m->LOSS.ensure(sizeof(double)))) return r;
    m->cap_rows = n;
    return MIRAGE_OK;
}

template <int BN>
int gemm_tc(const __nv_bfloat16* A, long sam, long sak, const __nv_bfloat16* B, long sbk, long sbn, float* C, int ldc,
            int M, int N, int K, cudaStream_t st) {
    constexpr int smem = tc_smem_bytes<BN>();
    const dim3 grid((unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)((N + BN - 1) / BN));
    k_gemm_tc<BN><<<grid, 128, smem, st>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K);
    MCK(cudaGetLastError());
    return MIRAGE_OK;
}

// raises the product kernels' shared-memory limit on the current device
// (once per network, outside any stream capture)
int gemm_setup() {
    MCK(cudaFuncSetAttribute(k_gemm_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes<16>()));
    MCK(cudaFuncSetAttribute(k_gemm_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes<32>()));
    MCK(cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes<64>()));
    return MIRAGE_OK;
}

// the N tile: 16 or 32 for the narrow output layer, else 64 columns (the
// 256-wide layers run in four tiles: more CTAs, each with a shorter
// staging pass)
int gemm(const __nv_bfloat16* A, long sam, long sak, const __nv_bfloat16* B, long sbk, long sbn, float* C, int ldc,
         int M, int N, int K, cudaStream_t st) {
    if (M <= 0 || N <= 0) return MIRAGE_OK;
    if (N <= 16) return gemm_tc<16>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, st);
    if (N <= 32) return gemm_tc<32>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, st);
    return gemm_tc<64>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, st);
}

// forward pass storing Z (FP32) and A (BF16); Y (FP32) written to y.  With
// idx, batch row j is row idx[j] of x.
int forward_pass(mirage_mlp* m, const float* x, int n, float* y, cudaStream_t st, const int* idx = nullptr) {
    int r;
    if ((r = ensure_batch(m, n))) return r;
    float* Z = (float*)m->Z.p;
    __nv_bfloat16* A = (__nv_bfloat16*)m->A.p;
    const float* P = (const float*)m->P.p;
    const __nv_bfloat16* PH = (const __nv_bfloat16*)m->PH.p;
    k_to_bf16<<<blocks((long)n * m->dims[0], 256), 256, 0, st>>>(x, idx, m->dims[0], A, (long)n * m->dims[0]);
    for (int l = 1; l <= m->L; ++l) {
        const int in = m->dims[l - 1], out = m->dims[l];
        // Z_l = A_{l-1} W_l^T : A(m, k) = A[m in + k], B(k, j) = W[j in + k]
        if ((r = gemm(A + m->a_off[l - 1], in, 1, PH + m->w_off[l - 1], 1, in, Z + m->z_off[l], out, n, out, in, st)))
            return r;
        const bool hidden = l < m->L;
        k_bias_act<<<blocks((long)n * out, 256), 256, 0, st>>>(Z + m->z_off[l], P + m->b_off[l - 1], n, out, hidden,
                                                               A + m->a_off[l], y);
        MCK(cudaGetLastError());
    }
    return MIRAGE_OK;
}

// gradients of the MSE into m->G (and the loss into m->LOSS if wanted)
int backward_pass(mirage_mlp* m, const float* x, const float* tgt, int n, float* yscratch, bool want_loss,
                  cudaStream_t st, const int* idx = nullptr) {
    int r;
    if ((r = forward_pass(m, x, n, yscratch, st, idx))) return r;
    float* Z = (float*)m->Z.p;
    __nv_bfloat16* A = (__nv_bfloat16*)m->A.p;
    float* DZ = (float*)m->DZ.p;
    __nv_bfloat16* DZH = (__nv_bfloat16*)m->DZH.p;
    float* DA = (float*)m->DA.p;
    float* G = (float*)m->G.p;
    const __nv_bfloat16* PH = (const __nv_bfloat16*)m->PH.p;
    double* loss = want_loss ? (double*)m->LOSS.p : nullptr;
    if (loss) MCK(cudaMemsetAsync(loss, 0, sizeof(double), st));
    const int outL = m->dims[m->L];
    k_loss_grad<<<blocks((long)n * outL, 256), 256, 0, st>>>(yscratch, tgt, idx, outL, (long)n * outL, DZ, DZH,
                                                             loss);
    MCK(cudaGetLastError());
    for (int l = m->L; l >= 1; --l) {
        const int in = m->dims[l - 1], out = m->dims[l];
        // dW_l = dZ^T A_{l-1}: [out x in];  A(mm, k) = dZ[k out + mm], B(k, j) = A_{l-1}[k in + j]
        if ((r = gemm(DZH, 1, out, A + m->a_off[l - 1], in, 1, G + m->w_off[l - 1], in, out, in, n, st))) return r;
        k_colsum<<<blocks(out, 128), 128, 0, st>>>(DZ, n, out, G + m->b_off[l - 1]);
        MCK(cudaGetLastError());
        if (l > 1) {
            // dA_{l-1} = dZ W_l: A(mm, k) = dZ[mm out + k], B(k, j) = W[k in + j]
            if ((r = gemm(DZH, out, 1, PH + m->w_off[l - 1], in, 1, DA, in, n, in, out, st))) return r;
            k_act_back<<<blocks((long)n * in, 256), 256, 0, st>>>(DA, Z + m->z_off[l - 1], (long)n * in, DZ, DZH);
            MCK(cudaGetLastError());
        }
    }
    return MIRAGE_OK;
}

// deterministic host RNG (splitmix64 + Box-Muller) for the initial weights
struct HostRng {
    unsigned long long s;
    unsigned long long next() {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

}  // namespace

extern "C" {

int mirage_mlp_create(mirage_mlp_t** out, int device, int n_layers, const int* dims, unsigned long long seed) {
    if (!out || n_layers < 1 || n_layers > 16 || !dims) return mlp_fail(MIRAGE_ERR_ARG, "mlp_create: bad arguments");
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > 4096) return mlp_fail(MIRAGE_ERR_ARG, "mlp_create: layer width out of range");
    MCK(cudaSetDevice(device));
    if (const int rs = gemm_setup()) return rs;
    mirage_mlp* m = new mirage_mlp();
    m->device = device;
    m->L = n_layers;
    m->dims.assign(dims, dims + n_layers + 1);
    long off = 0;
    for (int l = 0; l < n_layers; ++l) {
        m->w_off.push_back(off);
        off += (long)dims[l + 1] * dims[l];
        m->b_off.push_back(off);
        off += dims[l + 1];
    }
    m->n_params = off;
    int r = 0;
    if ((r = m->P.ensure(sizeof(float) * off)) || (r = m->PH.ensure(sizeof(__nv_bfloat16) * off)) ||
        (r = m->M.ensure(sizeof(float) * off)) || (r = m->V.ensure(sizeof(float) * off)) ||
        (r = m->G.ensure(sizeof(float) * off)) || (r = m->ISW.ensure(off))) {
        delete m;
        return r;
    }
    // He-style initial weights (std sqrt(2 / fan_in)), zero biases
    std::vector<float> h(off, 0.f);
    std::vector<unsigned char> isw(off, 0);
    HostRng rng{seed};
    for (int l = 0; l < n_layers; ++l) {
        const double sd = std::sqrt(2.0 / dims[l]);
        for (long i = 0; i < (long)dims[l + 1] * dims[l]; ++i) {
            h[m->w_off[l] + i] = (float)(sd * rng.normal());
            isw[m->w_off[l] + i] = 1;
        }
    }
    if (cudaMemcpy(m->ISW.p, isw.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete m;
        return mlp_fail(MIRAGE_ERR_CUDA, "mlp_create: upload failed");
    }
    *out = m;
    return mirage_mlp_set_params(m, h.data(), off);
}

int mirage_mlp_destroy(mirage_mlp_t* m) {
    if (!m) return MIRAGE_OK;
    cudaSetDevice(m->device);
    Buf* bufs[] = {&m->P,  &m->PH,  &m->M,  &m->V,    &m->G,   &m->ISW,  &m->Z,
                   &m->A,  &m->DZ,  &m->DZH, &m->DA,  &m->LOSS, &m->IDX, &m->DSTEP};
    for (Buf* b : bufs) b->release();
    if (m->cap) cudaStreamDestroy(m->cap);
    delete m;
    return MIRAGE_OK;
}

long mirage_mlp_num_params(const mirage_mlp_t* m) { return m ? m->n_params : 0; }

int mirage_mlp_set_params(mirage_mlp_t* m, const float* host_params, long n) {
    if (!m || !host_params || n != m->n_params) return mlp_fail(MIRAGE_ERR_ARG, "mlp_set_params: size mismatch");
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpy(m->P.p, host_params, sizeof(float) * n, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->M.p, 0, sizeof(float) * n));
    MCK(cudaMemset(m->V.p, 0, sizeof(float) * n));
    k_params_bf16<<<blocks(n, 256), 256>>>((const float*)m->P.p, (__nv_bfloat16*)m->PH.p, n);
    MCK(cudaGetLastError());
    MCK(cudaDeviceSynchronize());
    m->step = 0;
    return MIRAGE_OK;
}

int mirage_mlp_get_params(const mirage_mlp_t* m, float* host_params, long n) {
    if (!m || !host_params || n != m->n_params) return mlp_fail(MIRAGE_ERR_ARG, "mlp_get_params: size mismatch");
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpy(host_params, m->P.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return MIRAGE_OK;
}

int mirage_mlp_forward(mirage_mlp_t* m, const float* x, int n, float* y, void* stream) {
    if (!m || !x || !y || n < 0) return mlp_fail(MIRAGE_ERR_ARG, "mlp_forward: bad arguments");
    if (n == 0) return MIRAGE_OK;
    MCK(cudaSetDevice(m->device));
    return forward_pass(m, x, n, y, reinterpret_cast<cudaStream_t>(stream));
}

int mirage_mlp_grad(mirage_mlp_t* m, const float* x, const float* t, int n, float* grad, double* loss, float* y,
                    void* stream) {
    if (!m || !x || !t || !y || n < 1) return mlp_fail(MIRAGE_ERR_ARG, "mlp_grad: bad arguments");
    MCK(cudaSetDevice(m->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int r = backward_pass(m, x, t, n, y, loss != nullptr, st);
    if (r) return r;
    if (grad) MCK(cudaMemcpyAsync(grad, m->G.p, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice, st));
    if (loss) MCK(cudaMemcpyAsync(loss, m->LOSS.p, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return MIRAGE_OK;
}

int mirage_mlp_train_step(mirage_mlp_t* m, const float* x, const float* t, int n, float lr, double* loss, float* y,
                          void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int r = mirage_mlp_grad(m, x, t, n, nullptr, loss, y, stream);
    if (r) return r;
    m->step += 1;
    const float c1 = 1.f - std::pow(m->b1, (float)m->step), c2 = 1.f - std::pow(m->b2, (float)m->step);
    k_adam<<<blocks(m->n_params, 256), 256, 0, st>>>((float*)m->P.p, (const float*)m->G.p, (float*)m->M.p,
                                                     (float*)m->V.p, m->n_params, lr, m->b1, m->b2, m->eps, c1, c2,
                                                     (__nv_bfloat16*)m->PH.p, (const unsigned char*)m->ISW.p);
    MCK(cudaGetLastError());
    return MIRAGE_OK;
}

int mirage_mlp_train(mirage_mlp_t* m, const float* x, const float* t, int n, int steps, int batch, float lr,
                     unsigned long long seed, void* stream) {
    if (!m || !x || !t || n < 1 || steps < 0 || batch < 1 || batch > (1 << 20))
        return mlp_fail(MIRAGE_ERR_ARG, "mlp_train: bad arguments");
    if (steps == 0) return MIRAGE_OK;
    MCK(cudaSetDevice(m->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int r;
    // every buffer the step touches exists before the capture (no allocation inside it)
    if ((r = ensure_batch(m, batch)) || (r = m->IDX.ensure(sizeof(int) * (size_t)batch)) ||
        (r = m->DSTEP.ensure(sizeof(long long))))
        return r;
    if (!m->cap) MCK(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
    long long* dstep = (long long*)m->DSTEP.p;
    int* idx = (int*)m->IDX.p;
    float* y = (float*)m->DA.p;  // the step's forward output (DA is free until the backward pass)
    const long long s0 = m->step;
    MCK(cudaMemcpyAsync(dstep, &s0, sizeof(long long), cudaMemcpyHostToDevice, st));

    // one training step: draw rows, forward, MSE gradient, Adam; captured once
    cudaGraph_t graph = nullptr;
    MCK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    k_sample_rows<<<blocks(batch, 256), 256, 0, m->cap>>>(idx, batch, n, seed, dstep);
    r = backward_pass(m, x, t, batch, y, false, m->cap, idx);
    if (!r) {
        k_adam_dev<<<blocks(m->n_params, 256), 256, 0, m->cap>>>(
            (float*)m->P.p, (const float*)m->G.p, (float*)m->M.p, (float*)m->V.p, m->n_params, lr, m->b1, m->b2,
            m->eps, dstep, (__nv_bfloat16*)m->PH.p, (const unsigned char*)m->ISW.p);
        k_step_inc<<<1, 1, 0, m->cap>>>(dstep);
    }
    const cudaError_t ec = cudaStreamEndCapture(m->cap, &graph);
    if (r) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (ec != cudaSuccess || !graph)
        return mlp_fail(MIRAGE_ERR_CUDA, std::string("mlp_train: capture failed: ") + cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
        return mlp_fail(MIRAGE_ERR_CUDA, std::string("mlp_train: instantiate failed: ") + cudaGetErrorString(ei));
    cudaError_t el = cudaSuccess;
    for (int k = 0; k < steps && el == cudaSuccess; ++k) el = cudaGraphLaunch(exec, st);
    cudaGraphExecDestroy(exec);
    if (el != cudaSuccess)
        return mlp_fail(MIRAGE_ERR_CUDA, std::string("mlp_train: graph launch failed: ") + cudaGetErrorString(el));
    m->step += steps;
    return MIRAGE_OK;
}

const char* mirage_mlp_last_error(void) { return g_mlp_err.c_str(); }

}  // extern "C"
