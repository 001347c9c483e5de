// Allocation-free forward model: mirage_forward_noalloc.
//
// Some callers cannot let a library allocate device memory: a host
// framework that owns the whole device-memory budget through its own pool,
// a latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device, or code that must not grow its footprint after start-up.  This
// entry point runs the same ray-trace and forward kernels as mirage_forward
// but takes all its scratch from one fixed array in the library's own
// device memory (a file-scope __device__ array), so it never calls
// cudaMalloc, cudaFree or any other allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "internal.h"

using namespace mirage;

namespace {

// Scratch of every call of mirage_forward_noalloc on this device.  Every
// device that loads the library holds these bytes until the process exits.
constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB
constexpr int kNoAllocGrid = 32;                    // CTAs of the forward kernel
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of the array per device ordinal, looked up on the first
// call on that device.  The cache lives as long as the process: after a
// cudaDeviceReset the module is loaded again and the address may change,
// so a caller that resets a device must not call this entry point again on
// it in the same process.
void* g_scratch_ptr[kMaxDevices] = {};

// per calling thread, like the library's other error strings
thread_local char g_err[256] = "";

int fail(int code, const char* msg) {
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

// Device address of the scratch array for the current device (set up once
// per device: the array's name is only a host-side stand-in in host code).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(MIRAGE_ERR_CUDA, "forward_noalloc: no current CUDA device");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail(MIRAGE_ERR_CUDA, "forward_noalloc: cudaGetSymbolAddress failed");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MIRAGE_OK;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Writes the problem descriptor and the candidate index 0 into the array.
// The descriptor travels as a kernel parameter, which the launch copies, so
// no host buffer has to outlive the call.
template <typename T>
__global__ void k_put_problem(const Prob<T> P, Prob<T>* dst, int* cand) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *dst = P;
        *cand = 0;
    }
}

template <typename T>
int forward_noalloc_impl(const mirage_problem_t* prob, const double* lens, const void* s, int n_src, void* model,
                         double* chi2, int* status, cudaStream_t st) {
    constexpr int prec = sizeof(T) == 4 ? 0 : 1;
    if (!prob || !lens || !s || !chi2 || n_src < 0)
        return fail(MIRAGE_ERR_ARG, "forward_noalloc: null pointer or negative n_src");
    if (geometry_ok(prob->geom) != MIRAGE_OK || !prob->d || !prob->sigma || !prob->mask || !prob->psf)
        return fail(MIRAGE_ERR_ARG, "forward_noalloc: bad problem");
    if (n_src == 0) return MIRAGE_OK;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MIRAGE_OK) return rc;

    const Prob<T> P = problem_layout<T>(*prob);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((long long)P.ncells * 4 > max_smem - 2048)
        return fail(MIRAGE_ERR_UNSUPPORTED, "forward_noalloc: source grid too large for the ray-trace kernel");

    // carve the fixed array: problem, rays, cell starts, weights, image slab
    const long long sE = P.nrays, sInv = P.nrays, sCst = (P.ncells + 1 + 3) / 4 * 4, sPad = (P.plen + 3) / 4 * 4;
    const int grid = std::min(n_src, kNoAllocGrid);
    const long long stride = (P.plen + 63) / 64 * 64;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(bytes);
        return o;
    };
    const size_t o_prob = take(sizeof(Prob<T>) + sizeof(int));
    const size_t o_E = take(sizeof(Entry<T>) * sE);
    const size_t o_E64 = sizeof(T) == 4 ? take(sizeof(Entry<double>) * sE) : o_E;
    const size_t o_Et = take(sizeof(Entry<double>) * sE);
    const size_t o_inv = take(sizeof(int) * sInv);
    const size_t o_cst = take(sizeof(int) * sCst);
    const size_t o_swp = take(sizeof(T) * sPad);
    const size_t o_dpad = take(sizeof(T) * sPad);
    const size_t o_nent = take(sizeof(int));
    const size_t o_cstat = take(sizeof(int));
    const size_t o_slab = take(sizeof(T) * stride * grid);
    if (off > kNoAllocBytes) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "forward_noalloc: problem needs %zu bytes of scratch, the fixed array holds %zu "
                      "(use mirage_forward for larger images)",
                      off, kNoAllocBytes);
        return fail(MIRAGE_ERR_UNSUPPORTED, msg);
    }
    char* b = static_cast<char*>(base);

    // problem descriptor and its candidate index (0) into the array
    k_put_problem<T><<<1, 32, 0, st>>>(P, reinterpret_cast<Prob<T>*>(b + o_prob),
                                       reinterpret_cast<int*>(b + o_prob + sizeof(Prob<T>)));
    if (cudaGetLastError() != cudaSuccess)
        return fail(MIRAGE_ERR_CUDA, "forward_noalloc: writing the problem descriptor failed");

    CandScratch<T> cs;
    cs.E = reinterpret_cast<Entry<T>*>(b + o_E);
    cs.E64 = reinterpret_cast<Entry<double>*>(b + o_E64);
    cs.Etmp = reinterpret_cast<Entry<double>*>(b + o_Et);
    cs.inv = reinterpret_cast<int*>(b + o_inv);
    cs.cst = reinterpret_cast<int*>(b + o_cst);
    cs.swp = reinterpret_cast<T*>(b + o_swp);
    cs.dpad = reinterpret_cast<T*>(b + o_dpad);
    cs.nent = reinterpret_cast<int*>(b + o_nent);
    cs.cstat = reinterpret_cast<int*>(b + o_cstat);
    cs.sE = sE;
    cs.sInv = sInv;
    cs.sCst = sCst;
    cs.sPad = sPad;
    const Prob<T>* dprob = reinterpret_cast<const Prob<T>*>(b + o_prob);
    const int* dcand = reinterpret_cast<const int*>(b + o_prob + sizeof(Prob<T>));

    // the ray trace zero-fills the weights and cell counts it builds, and
    // the forward kernel zero-fills its image slab, so no state of an
    // earlier call survives into this one
    const KernelTable& tb = kernel_table();
    const void* rt = tb.raytrace[prec];
    const size_t rt_smem = (size_t)P.ncells * 4;
    if (cudaFuncSetAttribute(rt, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 2048) != cudaSuccess)
        return fail(MIRAGE_ERR_CUDA, "forward_noalloc: cudaFuncSetAttribute failed");
    int cand0 = 0, nc = 1;
    void* a1[] = {(void*)&dprob, (void*)&dcand, (void*)&lens, &cand0, &nc, &cs};
    if (cudaLaunchKernel(rt, dim3(1), dim3(NTHREADS), a1, rt_smem, st) != cudaSuccess)
        return fail(MIRAGE_ERR_CUDA, "forward_noalloc: ray-trace launch failed");
    const void* fn = (P.K < MAX_K && tb.fwd[prec][P.K]) ? tb.fwd[prec][P.K] : tb.fwd[prec][0];
    const size_t smem = align_up<T>(sizeof(T) * P.K * P.kp, 16) + 2 * 33 * sizeof(double) + 16;
    const T* S = reinterpret_cast<const T*>(s);
    T* M = reinterpret_cast<T*>(model);
    T* slab = reinterpret_cast<T*>(b + o_slab);
    long long sstr = stride;
    void* a2[] = {(void*)&dprob, &cs, (void*)&S, &n_src, &M, &chi2, &slab, &sstr, &status};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(NTHREADS), a2, smem, st) != cudaSuccess)
        return fail(MIRAGE_ERR_CUDA, "forward_noalloc: forward launch failed");
    return MIRAGE_OK;
}

}  // namespace

extern "C" {

int mirage_forward_noalloc(int precision, const mirage_problem_t* prob, const double* lens, const void* s,
                           int n_src, void* model, double* chi2, int* status, void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (precision == MIRAGE_FP32) return forward_noalloc_impl<float>(prob, lens, s, n_src, model, chi2, status, st);
    if (precision == MIRAGE_FP64) return forward_noalloc_impl<double>(prob, lens, s, n_src, model, chi2, status, st);
    return fail(MIRAGE_ERR_ARG, "forward_noalloc: precision must be MIRAGE_FP32 or MIRAGE_FP64");
}

const char* mirage_noalloc_last_error(void) { return g_err; }

size_t mirage_noalloc_capacity(void) { return kNoAllocBytes; }

}  // extern "C"
