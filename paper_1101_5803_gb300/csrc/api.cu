// C ABI of the lens-inversion inner loop: context, argument checks, scratch
// management, work-item planning, launches and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <initializer_list>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mirage.h"
#include "fast.cuh"
#include "forward.cuh"
#include "iterlc.cuh"
#include "kernels.cuh"
#include "table.h"

using namespace mirage;

namespace {

thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                        \
            return e_ == cudaErrorMemoryAllocation ? MIRAGE_ERR_NOMEM : MIRAGE_ERR_CUDA; \
        }                                                                               \
    } while (0)

const KernelTable& table() {
    static KernelTable t = [] {
        KernelTable k;
        std::memset(&k, 0, sizeof(k));
        fill_f32_k5(k);
        fill_f32_k7(k);
        fill_f32_k9(k);
        fill_f32_k11(k);
        fill_f32_k15(k);
        fill_f32_k21(k);
        fill_f32_gen(k);
        fill_f64(k);
        fill_fast(k);
        fill_iter(k);
        fill_fwd_band(k);
        return k;
    }();
    return t;
}

// grow-only device buffer owned by the context
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    int ensure(size_t bytes) {
        if (bytes <= n) return MIRAGE_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
            p = nullptr;
            return MIRAGE_ERR_NOMEM;
        }
        n = want;
        return MIRAGE_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <typename U>
    U* as() const {
        return reinterpret_cast<U*>(p);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    DevBuf probs, meta;  // this graph's own copy of the launch metadata
};

}  // namespace

struct mirage_ctx {
    int device = 0;
    int precision = MIRAGE_FP32;
    int sm_count = 0;
    int max_smem = 0;
    int max_smem_sm = 0;
    int last_launches = 0;
    int reserved = 0;  // CTA slots the CGLS launches leave free (mirage_set_reserved_slots)
    // scratch
    DevBuf E, E64, Etmp, inv, cst, swp, dpad, nent, cstat, X, istat, slab, probs, cand_prob, items, counters;
    DevBuf stage;  // MIRAGE_MEM_HOST staging
    DevBuf fE, fE64, fEtmp, finv, fcst, fswp, fdpad, fnent, fcstat, fslab, fprob, fcand, fpix;
    DevBuf rt_cursor;  // per-cell cursors of the parallel ray placement
    DevBuf spec;       // PSF spectra of the FFT-convolution problems (FP64, then FP32)
    // pinned staging of the per-call uploads (problem descriptors, item
    // tables): the copies stay asynchronous; the event guards reuse
    void* pin = nullptr;
    size_t pin_n = 0;
    cudaEvent_t pin_ev = nullptr;
    bool pin_pending = false;
    std::map<std::string, GraphEntry> graphs;
    std::map<const void*, int> smem_set;  // kernel -> dynamic smem attribute set
    cudaStream_t cap_stream = nullptr;   // graphs are captured here and launched on the caller's stream
    cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};  // concurrent kernel groups
    cudaEvent_t fork_ev = nullptr, join_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // phase timing (opts.threads < 0)
    DevBuf clk;                                                  // per-phase SM clocks (opts.threads == -2)
    int timed = 0;
    std::vector<void*> scratch_seen;     // scratch pointers the cached graphs were captured with
};

// CTAs of a persistent CGLS launch: per_sm on every SM, less the slots the
// caller reserved for concurrent work on other streams (at least one)
static long long cgls_slots(const mirage_ctx* ctx, int per_sm) {
    return std::max<long long>(1, (long long)per_sm * ctx->sm_count - ctx->reserved);
}

// a PSF tap as the fast kernel's parameter: as is, or rounded to TF32
// (nearest, ties away from zero: the cvt.rna.tf32 rule) for the TF32
// precision variant
static float tap_value(float t, bool tf32) {
    if (!tf32) return t;
    unsigned u;
    std::memcpy(&u, &t, sizeof(u));
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & ~0x1fffu;
    float r;
    std::memcpy(&r, &u, sizeof(r));
    return r;
}

// relative CG iteration count of lambda index k of an n-point ascending
// grid: measured counts scale like lambda^-0.37, and the grids span about six
// decades log-spaced, so the count grows by 10^(2.2 / (n - 1)) per step
// towards small lambda
static double chain_weight(int n, int k) {
    return n > 1 ? std::pow(10.0, 2.2 * (double)(n - 1 - k) / (double)(n - 1)) : 1.0;
}

namespace {
void drop_graphs(mirage_ctx* ctx) {
    for (auto& kv : ctx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        kv.second.probs.release();
        kv.second.meta.release();
    }
    ctx->graphs.clear();
}
}  // namespace

namespace {

template <typename T>
constexpr int prec_of() {
    return sizeof(T) == 4 ? 0 : 1;
}

int check_geom(const mirage_geom_t& g) {
    if (g.nx < 1 || g.ny < 1 || g.nx > 4096 || g.ny > 4096) return MIRAGE_ERR_ARG;
    if (g.sx < 2 || g.sy < 2 || (long long)g.sx * g.sy > (1 << 20)) return MIRAGE_ERR_ARG;
    if (!(g.pix > 0) || !(g.sxmax > g.sxmin) || !(g.symax > g.symin)) return MIRAGE_ERR_ARG;
    if (g.kpsf < 1 || g.kpsf > MIRAGE_MAX_KPSF || (g.kpsf % 2) == 0) return MIRAGE_ERR_ARG;
    if (g.subpix < 1 || g.subpix > 8) return MIRAGE_ERR_ARG;
    if (g.reg < 0 || g.reg > 2) return MIRAGE_ERR_ARG;
    if (g.interp != MIRAGE_INTERP_BILINEAR && g.interp != MIRAGE_INTERP_NEAREST && g.interp != MIRAGE_INTERP_BICUBIC)
        return MIRAGE_ERR_ARG;
    if (!std::isfinite(g.cx) || !std::isfinite(g.cy)) return MIRAGE_ERR_ARG;
    return MIRAGE_OK;
}

template <typename T>
Prob<T> make_prob(const mirage_problem_t& mp, const void* d, const void* sigma, const void* mask, const void* psf) {
    const mirage_geom_t& g = mp.geom;
    Prob<T> P;
    std::memset(&P, 0, sizeof(P));
    P.nx = g.nx;
    P.ny = g.ny;
    P.npix = g.nx * g.ny;
    P.sx = g.sx;
    P.sy = g.sy;
    P.ns = g.sx * g.sy;
    P.reg = g.reg;
    P.interp = g.interp;
    P.nreg = g.reg == MIRAGE_REG_GRADIENT ? 2 * P.ns : P.ns;
    P.K = g.kpsf;
    P.hk = (g.kpsf - 1) / 2;
    P.kp = (g.kpsf + 3) & ~3;
    P.n_sub = g.subpix;
    P.Np = g.subpix * g.subpix;
    P.nrays = P.npix * P.Np;
    P.ncx = g.sx - 1;
    P.ncells = (g.sx - 1) * (g.sy - 1);
    P.tiles_x = (g.nx + TILE - 1) / TILE;
    P.tiles_y = (g.ny + TILE - 1) / TILE;
    P.ntiles = P.tiles_x * P.tiles_y;
    const int VW = 16 / (int)sizeof(T);
    P.xoff = (P.hk + VW - 1) / VW * VW;
    const int sh = P.xoff - P.hk;
    const int nvw = (TILE + g.kpsf - 1 + sh + VW - 1) / VW * VW;
    P.Wp = std::max((P.tiles_x - 1) * TILE + nvw, P.xoff + g.nx + P.hk);
    P.Wp = (P.Wp + VW - 1) / VW * VW;
    P.Hp = P.tiles_y * TILE + g.kpsf - 1;
    P.plen = P.Wp * P.Hp;
    P.pix = g.pix;
    P.cx = g.cx;
    P.cy = g.cy;
    P.sub0 = (0.5 / g.subpix - 0.5) * g.pix;
    P.subd = g.pix / g.subpix;
    P.hx = (g.sxmax - g.sxmin) / g.sx;
    P.hy = (g.symax - g.symin) / g.sy;
    P.c0x = g.sxmin + 0.5 * P.hx;
    P.c0y = g.symin + 0.5 * P.hy;
    P.invNp = (T)(1.0 / P.Np);
    P.d = reinterpret_cast<const T*>(d);
    P.sigma = reinterpret_cast<const T*>(sigma);
    P.mask = reinterpret_cast<const uint8_t*>(mask);
    P.psf = reinterpret_cast<const T*>(psf);
    return P;
}

int set_smem(mirage_ctx* ctx, const void* fn, size_t bytes) {
    auto it = ctx->smem_set.find(fn);
    if (it == ctx->smem_set.end()) {
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, fn));
        const int dyn_max = ctx->max_smem - (int)fa.sharedSizeBytes;
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
        it = ctx->smem_set.emplace(fn, dyn_max).first;
    }
    if ((long long)bytes > it->second) {
        set_error("work item needs %zu B of dynamic shared memory (limit %d)", bytes, it->second);
        return MIRAGE_ERR_UNSUPPORTED;
    }
    return MIRAGE_OK;
}

const void* pick_cgls(int prec, int place, int K) {
    const KernelTable& t = table();
    const void* f = K < MAX_K ? t.cgls[prec][place][K] : nullptr;  // wider PSFs: the runtime-K kernel
    return f ? f : t.cgls[prec][place][0];
}

// placement of the general kernel's work buffers for one problem
template <typename T>
int pick_place(const mirage_ctx* ctx, const Prob<T>& P, int want = 0) {
    if (P.fft_m) return PLACE_GLOBAL;  // the FFT path lives in the runtime-K global-memory kernel
    // a requested placement (mirage_opts_t.place: 1 SMEM, 2 MID, 3 GLOBAL,
    // 4 GLOBAL with two CTAs per SM) where it fits
    if (want == 1 && smem_bytes<T>(P, PLACE_SMEM) <= (size_t)ctx->max_smem) return PLACE_SMEM;
    if (want == 2 && sizeof(T) == 4 && smem_bytes<T>(P, PLACE_MID) <= (size_t)ctx->max_smem) return PLACE_MID;
    if (want == 3) return PLACE_GLOBAL;
    if (want == 4) {
        const KernelTable& t = table();
        if (sizeof(T) == 4 && (t.cgls[0][PLACE_GLOBAL2][P.K < MAX_K ? P.K : 0] || t.cgls[0][PLACE_GLOBAL2][0]) &&
            2 * (long long)smem_bytes<T>(P, PLACE_GLOBAL) <= ctx->max_smem_sm - 2048)
            return PLACE_GLOBAL2;
        return PLACE_GLOBAL;
    }
    if (want == 5 && sizeof(T) == 4) {
        const KernelTable& t = table();
        if ((t.cgls[0][PLACE_MID2][P.K < MAX_K ? P.K : 0] || t.cgls[0][PLACE_MID2][0]) &&
            2 * ((long long)smem_bytes<T>(P, PLACE_MID) + 1024) <= ctx->max_smem_sm)
            return PLACE_MID2;
    }
    if (smem_bytes<T>(P, PLACE_SMEM) <= (size_t)ctx->max_smem) return PLACE_SMEM;
    if (sizeof(T) == 4 && smem_bytes<T>(P, PLACE_MID) <= (size_t)ctx->max_smem) return PLACE_MID;
    // all in the slab: two CTAs per SM where that kernel is compiled for the
    // problem's PSF width (FP32; 1.47x faster at 256 x 256 with a 21 x 21 PSF,
    // where one 253-register CTA per SM could not hide the slab's latency)
    if (sizeof(T) == 4 && P.K < MAX_K && table().cgls[0][PLACE_GLOBAL2][P.K] &&
        2 * (long long)smem_bytes<T>(P, PLACE_GLOBAL) <= ctx->max_smem_sm - 2048)
        return PLACE_GLOBAL2;
    return PLACE_GLOBAL;
}

// FFT convolution of a problem's lambda-grid solves: forced by variant 5,
// never with variant 6 (direct convolution at any width), otherwise for PSFs
// of FFT_AUTO_K taps and wider.  The grid side is the
// smallest power of two >= max(nx, ny) + (K - 1) / 2 (at least 16, at most
// 1024); problems whose FFT buffers do not fit in shared memory keep the
// direct convolution.
constexpr int FFT_AUTO_K = 23;  // the first width without a compiled direct kernel; measured crossover 21..25

template <typename T>
void plan_fft(const mirage_ctx* ctx, Prob<T>& P, int variant) {
    P.fft_m = 0;
    P.fft_log = 0;
    if (variant == 6 || (variant != 5 && P.K < FFT_AUTO_K)) return;
    const int M = std::max(16, fft_size_for(std::max(P.nx, P.ny) + P.hk));
    if (M > 1024) return;
    Prob<T> Q = P;
    Q.fft_m = M;
    if (smem_bytes<T>(Q, PLACE_GLOBAL) > (size_t)ctx->max_smem) return;
    P.fft_m = M;
    while ((1 << P.fft_log) < M) ++P.fft_log;
}

const void* pick_fwd(int prec, int K) {
    const KernelTable& t = table();
    const void* f = K < MAX_K ? t.fwd[prec][K] : nullptr;
    return f ? f : t.fwd[prec][0];
}

// two-CTA-per-SM kernel when the problem qualifies (FP32 contexts only)
template <typename T>
const void* pick_fast(mirage_ctx* ctx, const Prob<T>& P, int mode) {
    if (sizeof(T) != 4 || P.interp == MIRAGE_INTERP_BICUBIC) return nullptr;  // four-corner rays only
    const Prob<float>& Pf = *reinterpret_cast<const Prob<float>*>(&P);
    const size_t b = fast_smem_bytes(Pf);
    if (b == 0 || (long long)b > ctx->max_smem_sm / 2 - 1024 || Pf.K >= MAX_K) return nullptr;
    return table().fast[Pf.K][0][mode];
}

// fast-kernel arguments (FP32 contexts only; never called for double)
template <typename T>
void set_fast_args(FastArgs& fa, const CglsArgs<T>& A) {
    if constexpr (sizeof(T) == 4) std::memcpy(&fa.A, &A, sizeof(A));
}

template <typename T>
void fill_scratch(CandScratch<T>& cs, mirage_ctx* ctx, bool fwd, long long sE, long long sInv, long long sCst,
                  long long sPad) {
    cs.E = (fwd ? ctx->fE : ctx->E).as<Entry<T>>();
    cs.E64 = sizeof(T) == 8 ? reinterpret_cast<Entry<double>*>(cs.E) : (fwd ? ctx->fE64 : ctx->E64).as<Entry<double>>();
    cs.Etmp = (fwd ? ctx->fEtmp : ctx->Etmp).as<Entry<double>>();
    cs.inv = (fwd ? ctx->finv : ctx->inv).as<int>();
    cs.cst = (fwd ? ctx->fcst : ctx->cst).as<int>();
    cs.swp = (fwd ? ctx->fswp : ctx->swp).as<T>();
    cs.dpad = (fwd ? ctx->fdpad : ctx->dpad).as<T>();
    cs.nent = (fwd ? ctx->fnent : ctx->nent).as<int>();
    cs.cstat = (fwd ? ctx->fcstat : ctx->cstat).as<int>();
    cs.sE = sE;
    cs.sInv = sInv;
    cs.sCst = sCst;
    cs.sPad = sPad;
}

int launch(mirage_ctx* ctx, const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st) {
    CK(cudaLaunchKernel(fn, grid, block, args, smem, st));
    ctx->last_launches++;
    return MIRAGE_OK;
}

// asynchronous upload of small host arrays through the context's pinned
// staging buffer (a pageable source would make the copy synchronise the
// stream); the host arrays may go away as soon as this returns
struct UploadPart {
    void* dst;
    const void* src;
    size_t bytes;
};
int upload(mirage_ctx* ctx, cudaStream_t st, std::initializer_list<UploadPart> parts) {
    size_t total = 0;
    for (const UploadPart& u : parts) total += (u.bytes + 15) / 16 * 16;
    if (ctx->pin_pending) {
        CK(cudaEventSynchronize(ctx->pin_ev));  // the previous call's copies have left the buffer
        ctx->pin_pending = false;
    }
    if (!ctx->pin_ev) CK(cudaEventCreateWithFlags(&ctx->pin_ev, cudaEventDisableTiming));
    if (total > ctx->pin_n) {
        if (ctx->pin) cudaFreeHost(ctx->pin);
        ctx->pin = nullptr;
        ctx->pin_n = 0;
        const size_t want = std::max<size_t>(total, 1 << 16);
        if (cudaHostAlloc(&ctx->pin, want, cudaHostAllocDefault) != cudaSuccess) {
            ctx->pin = nullptr;
            set_error("cudaHostAlloc(%zu) failed", want);
            return MIRAGE_ERR_NOMEM;
        }
        ctx->pin_n = want;
    }
    size_t off = 0;
    for (const UploadPart& u : parts) {
        if (!u.bytes) continue;
        char* h = static_cast<char*>(ctx->pin) + off;
        std::memcpy(h, u.src, u.bytes);
        CK(cudaMemcpyAsync(u.dst, h, u.bytes, cudaMemcpyHostToDevice, st));
        off += (u.bytes + 15) / 16 * 16;
    }
    CK(cudaEventRecord(ctx->pin_ev, st));
    ctx->pin_pending = true;
    return MIRAGE_OK;
}

// ray trace of candidates [cand0, cand0 + n_cand): one CTA per candidate,
// or, for fewer candidates than SMs on large images, the split trace (many
// CTAs per candidate trace and count, one CTA per candidate places)
template <typename T>
int launch_raytrace(mirage_ctx* ctx, const Prob<T>* dprobs, const int* dcand, const double* d_lens, int cand0,
                    int n_cand, const CandScratch<T>& cs, long long max_cells, long long max_npix, cudaStream_t st);

#define TRY(x)                      \
    do {                            \
        int r_ = (x);               \
        if (r_ != MIRAGE_OK) return r_; \
    } while (0)

// staging of host arrays into one device block (MIRAGE_MEM_HOST)
struct Stager {
    std::vector<std::pair<size_t, std::pair<const void*, size_t>>> in;  // offset, (host ptr, bytes)
    std::vector<std::pair<size_t, std::pair<void*, size_t>>> out;
    size_t total = 0;
    size_t add_in(const void* h, size_t bytes) {
        const size_t o = total;
        total += (bytes + 255) / 256 * 256;
        if (h && bytes) in.push_back({o, {h, bytes}});
        return o;
    }
    size_t add_out(void* h, size_t bytes) {
        const size_t o = total;
        total += (bytes + 255) / 256 * 256;
        if (h && bytes) out.push_back({o, {h, bytes}});
        return o;
    }
};

template <typename T>
int launch_raytrace(mirage_ctx* ctx, const Prob<T>* dprobs, const int* dcand, const double* d_lens, int cand0,
                    int n_cand, const CandScratch<T>& cs, long long max_cells, long long max_npix, cudaStream_t st) {
    constexpr int prec = prec_of<T>();
    const KernelTable& tb = table();
    const size_t cells_smem = (size_t)max_cells * 4;
    if (n_cand < ctx->sm_count && max_npix >= 128 * 128) {
        const int chunk = 2 * NTHREADS;
        const int n_chunks = (int)((max_npix + chunk - 1) / chunk);
        CK(cudaMemsetAsync(cs.swp + (long long)cand0 * cs.sPad, 0, sizeof(T) * cs.sPad * n_cand, st));
        CK(cudaMemsetAsync(cs.dpad + (long long)cand0 * cs.sPad, 0, sizeof(T) * cs.sPad * n_cand, st));
        CK(cudaMemsetAsync(cs.cst + (long long)cand0 * cs.sCst, 0, sizeof(int) * cs.sCst * n_cand, st));
        CK(cudaMemsetAsync(cs.cstat + cand0, 0, sizeof(int) * n_cand, st));
        int c0 = cand0, ch = chunk;
        CandScratch<T> csv = cs;
        void* a1[] = {(void*)&dprobs, (void*)&dcand, (void*)&d_lens, &c0, &ch, &csv};
        TRY(launch(ctx, tb.rt_trace[prec], dim3(n_chunks, n_cand), dim3(NTHREADS), a1, 0, st));
        TRY(set_smem(ctx, tb.rt_place[prec], cells_smem));
        void* a2[] = {(void*)&dprobs, (void*)&dcand, (void*)&d_lens, &c0, &csv};
        TRY(launch(ctx, tb.rt_place[prec], dim3(n_cand), dim3(NTHREADS), a2, cells_smem, st));
        // one ray per pixel: parallel placement (the place kernel only scanned)
        TRY(ctx->rt_cursor.ensure(sizeof(int) * (size_t)cs.sCst * (cand0 + n_cand)));
        int* cur = ctx->rt_cursor.as<int>();
        long long cstr = cs.sCst;
        CK(cudaMemsetAsync(cur + (long long)cand0 * cstr, 0, sizeof(int) * cstr * n_cand, st));
        void* a3[] = {(void*)&dprobs, (void*)&dcand, (void*)&d_lens, &c0, &ch, &csv, (void*)&cur, &cstr};
        TRY(launch(ctx, tb.rt_scatter[prec], dim3(n_chunks, n_cand), dim3(NTHREADS), a3, 0, st));
        void* a4[] = {(void*)&dprobs, (void*)&dcand, (void*)&d_lens, &c0, &csv};
        return launch(ctx, tb.rt_sortcells[prec], dim3((unsigned)((max_cells + NTHREADS - 1) / NTHREADS), n_cand),
                      dim3(NTHREADS), a4, 0, st);
    }
    TRY(set_smem(ctx, tb.raytrace[prec], cells_smem));
    int c0 = cand0, nc = n_cand;
    CandScratch<T> csv = cs;
    void* args[] = {(void*)&dprobs, (void*)&dcand, (void*)&d_lens, &c0, &nc, &csv};
    return launch(ctx, tb.raytrace[prec], dim3(n_cand), dim3(NTHREADS), args, cells_smem, st);
}

// work item of the CGLS kernels: lambdas k_first..k_last of candidate c,
// solved in order by one CTA (see ChainPos)
inline int pack_chain(int c, int k_first, int k_last) { return (c * MAX_LAM + k_first) * MAX_LAM + k_last; }

template <typename T>
int eval_impl(mirage_ctx* ctx, const mirage_problem_t* probs, int n_probs, const double* lens, const int* prob_idx,
              int n_cand, const double* lambdas, const int* n_lam, int max_lam, const mirage_opts_t* opts,
              const void* warm_x, const int* lam_start, double* chi2, double* reg, int* iters, double* relres, int* item_status,
              int* corner, double* kappa, void* s_out, void* all_x, int* status, cudaStream_t st) {
    constexpr int prec = prec_of<T>();
    ctx->last_launches = 0;
    if (n_cand == 0) return MIRAGE_OK;
    if (!probs || n_probs < 1 || !lens || !prob_idx || !lambdas || !n_lam || !chi2 || !reg || !iters || !corner ||
        !status || max_lam < 1 || max_lam > MAX_LAM || n_cand < 0 || n_cand > INT_MAX / (MAX_LAM * MAX_LAM) - 1) {
        set_error("eval_batch: null pointer or size out of range");
        return MIRAGE_ERR_ARG;
    }
    const mirage_opts_t o = *opts;
    if (!(o.tol >= 0) || o.mode < 0 || o.mode > 1 || o.mem < 0 || o.mem > 1 || o.variant < 0 || o.variant > 7 ||
        !(o.inner_eta == 0.0 || (o.inner_eta >= 1e-4 && o.inner_eta <= 0.5)) || o.place < 0 || o.place > 5) {
        set_error("eval_batch: bad options");
        return MIRAGE_ERR_ARG;
    }
    for (int p = 0; p < n_probs; ++p) {
        if (check_geom(probs[p].geom) != MIRAGE_OK) {
            set_error("eval_batch: bad geometry of problem %d", p);
            return MIRAGE_ERR_ARG;
        }
        if (!probs[p].d || !probs[p].sigma || !probs[p].mask || !probs[p].psf) {
            set_error("eval_batch: null data pointer in problem %d", p);
            return MIRAGE_ERR_ARG;
        }
    }
    for (int c = 0; c < n_cand; ++c) {
        if (prob_idx[c] < 0 || prob_idx[c] >= n_probs || n_lam[c] < 1 || n_lam[c] > max_lam) {
            set_error("eval_batch: bad prob_idx / n_lam of candidate %d", c);
            return MIRAGE_ERR_ARG;
        }
    }
    const bool host = o.mem == MIRAGE_MEM_HOST;

    // sizes over the problems
    std::vector<Prob<T>> hp(n_probs);
    long long max_rays = 0, max_cells = 0, max_plen = 0, max_ns = 0, max_npix = 0;
    long long spec_stride = 0;
    for (int p = 0; p < n_probs; ++p) {
        hp[p] = make_prob<T>(probs[p], probs[p].d, probs[p].sigma, probs[p].mask, probs[p].psf);
        plan_fft<T>(ctx, hp[p], o.variant);
        if (hp[p].fft_m)
            spec_stride = std::max<long long>(spec_stride, (long long)((hp[p].fft_m >> 1) + 1) * hp[p].fft_m);
        max_npix = std::max<long long>(max_npix, hp[p].npix);
        max_rays = std::max<long long>(max_rays, hp[p].nrays);
        max_cells = std::max<long long>(max_cells, hp[p].ncells);
        max_plen = std::max<long long>(max_plen, hp[p].plen);
        max_ns = std::max<long long>(max_ns, hp[p].ns);
    }
    if ((long long)max_cells * 4 > ctx->max_smem - 2048) {
        set_error("source grid too large for the ray-trace kernel");
        return MIRAGE_ERR_UNSUPPORTED;
    }
    const long long sE = max_rays, sInv = max_rays, sCst = (max_cells + 1 + 3) / 4 * 4, sPad = (max_plen + 3) / 4 * 4;
    const long long nitems_all = (long long)n_cand * max_lam;

    // host staging: every array of the call goes through one device block
    const double* d_lens = lens;
    const double* d_lambdas = lambdas;
    const T* d_warm = reinterpret_cast<const T*>(warm_x);
    double *d_chi2 = chi2, *d_reg = reg, *d_relres = relres, *d_kappa = kappa;
    int *d_iters = iters, *d_istat = item_status, *d_corner = corner, *d_status = status;
    T *d_sout = reinterpret_cast<T*>(s_out), *d_allx = reinterpret_cast<T*>(all_x);
    if (host) {
        Stager sg;
        std::vector<size_t> po(4 * n_probs);
        for (int p = 0; p < n_probs; ++p) {
            const mirage_geom_t& g = probs[p].geom;
            const size_t np = (size_t)g.nx * g.ny;
            po[4 * p + 0] = sg.add_in(probs[p].d, np * sizeof(T));
            po[4 * p + 1] = sg.add_in(probs[p].sigma, np * sizeof(T));
            po[4 * p + 2] = sg.add_in(probs[p].mask, np);
            po[4 * p + 3] = sg.add_in(probs[p].psf, (size_t)g.kpsf * g.kpsf * sizeof(T));
        }
        const size_t o_lens = sg.add_in(lens, sizeof(double) * 7 * n_cand);
        const size_t o_lam = sg.add_in(lambdas, sizeof(double) * max_lam * n_cand);
        const size_t o_warm = sg.add_in(warm_x, warm_x ? sizeof(T) * nitems_all * max_ns : 0);
        const size_t o_chi2 = sg.add_out(chi2, sizeof(double) * nitems_all);
        const size_t o_reg = sg.add_out(reg, sizeof(double) * nitems_all);
        const size_t o_it = sg.add_out(iters, sizeof(int) * nitems_all);
        const size_t o_rr = sg.add_out(relres, relres ? sizeof(double) * nitems_all : 0);
        const size_t o_is = sg.add_out(item_status, item_status ? sizeof(int) * nitems_all : 0);
        const size_t o_cn = sg.add_out(corner, sizeof(int) * n_cand);
        const size_t o_kp = sg.add_out(kappa, kappa ? sizeof(double) * nitems_all : 0);
        const size_t o_so = sg.add_out(s_out, s_out ? sizeof(T) * n_cand * max_ns : 0);
        const size_t o_ax = sg.add_out(all_x, all_x ? sizeof(T) * nitems_all * max_ns : 0);
        const size_t o_st = sg.add_out(status, sizeof(int) * n_cand);
        TRY(ctx->stage.ensure(sg.total));
        char* base = ctx->stage.as<char>();
        for (auto& e : sg.in) CK(cudaMemcpyAsync(base + e.first, e.second.first, e.second.second, cudaMemcpyHostToDevice, st));
        for (int p = 0; p < n_probs; ++p)
            hp[p] = make_prob<T>(probs[p], base + po[4 * p], base + po[4 * p + 1], base + po[4 * p + 2],
                                 base + po[4 * p + 3]);
        d_lens = reinterpret_cast<const double*>(base + o_lens);
        d_lambdas = reinterpret_cast<const double*>(base + o_lam);
        d_warm = warm_x ? reinterpret_cast<const T*>(base + o_warm) : nullptr;
        d_chi2 = reinterpret_cast<double*>(base + o_chi2);
        d_reg = reinterpret_cast<double*>(base + o_reg);
        d_iters = reinterpret_cast<int*>(base + o_it);
        d_relres = relres ? reinterpret_cast<double*>(base + o_rr) : nullptr;
        d_istat = item_status ? reinterpret_cast<int*>(base + o_is) : nullptr;
        d_corner = reinterpret_cast<int*>(base + o_cn);
        d_kappa = kappa ? reinterpret_cast<double*>(base + o_kp) : nullptr;
        d_sout = s_out ? reinterpret_cast<T*>(base + o_so) : nullptr;
        d_allx = all_x ? reinterpret_cast<T*>(base + o_ax) : nullptr;
        d_status = reinterpret_cast<int*>(base + o_st);
        // run on device buffers, then copy back
        mirage_opts_t o2 = o;
        o2.mem = MIRAGE_MEM_DEVICE;
        o2.use_graph = 0;
        std::vector<mirage_problem_t> dp(probs, probs + n_probs);
        for (int p = 0; p < n_probs; ++p) {
            dp[p].d = base + po[4 * p];
            dp[p].sigma = base + po[4 * p + 1];
            dp[p].mask = reinterpret_cast<const uint8_t*>(base + po[4 * p + 2]);
            dp[p].psf = base + po[4 * p + 3];
        }
        TRY(eval_impl<T>(ctx, dp.data(), n_probs, d_lens, prob_idx, n_cand, d_lambdas, n_lam, max_lam, &o2, d_warm,
                         lam_start, d_chi2, d_reg, d_iters, d_relres, d_istat, d_corner, d_kappa, d_sout, d_allx, d_status,
                         st));
        const int nl = ctx->last_launches;
        for (auto& e : sg.out) CK(cudaMemcpyAsync(e.second.first, base + e.first, e.second.second, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx->last_launches = nl;
        return MIRAGE_OK;
    }

    // ---- device path
    TRY(ctx->E.ensure(sizeof(Entry<T>) * n_cand * sE));
    if (sizeof(T) == 4) TRY(ctx->E64.ensure(sizeof(Entry<double>) * n_cand * sE));
    TRY(ctx->Etmp.ensure(sizeof(Entry<double>) * n_cand * sE));
    TRY(ctx->inv.ensure(sizeof(int) * n_cand * sInv));
    TRY(ctx->cst.ensure(sizeof(int) * n_cand * sCst));
    TRY(ctx->swp.ensure(sizeof(T) * n_cand * sPad));
    TRY(ctx->dpad.ensure(sizeof(T) * n_cand * sPad));
    TRY(ctx->nent.ensure(sizeof(int) * n_cand));
    TRY(ctx->cstat.ensure(sizeof(int) * n_cand));
    if (!d_allx) TRY(ctx->X.ensure(sizeof(T) * nitems_all * max_ns));
    if (!d_istat) TRY(ctx->istat.ensure(sizeof(int) * nitems_all));
    T* dX = d_allx ? d_allx : ctx->X.as<T>();
    int* dIst = d_istat ? d_istat : ctx->istat.as<int>();

    // per-candidate kernel class and work items
    std::vector<int> cls_of(n_probs);
    struct Group {
        const void* fn;
        bool big;
        bool fast = false;
        int prob = -1;   // the single problem of the group, -2 if several
        int per_sm = 1;  // resident CTAs per SM
        double cost = 0.0;
        size_t smem = 0;
        long long slab = 0;
        std::vector<std::pair<double, int>> items;  // (sort key, packed)
    };
    std::map<std::pair<const void*, int>, Group> groups;
    std::vector<double> hlam;  // lambdas are device data: sort by index instead (ascending lambda = costlier)
    // kernel choice per problem: parameter taps need one PSF per launch
    std::vector<int> cands_of(n_probs, 0);
    for (int c = 0; c < n_cand; ++c) cands_of[prob_idx[c]]++;
    int n_used = 0;
    for (int p = 0; p < n_probs; ++p) n_used += cands_of[p] > 0;
    const int want = o.variant;
    auto choose = [&](const Prob<T>& P, int& mode, bool& fast) -> const void* {
        fast = false;
        mode = 0;
        if (want == 4 || want == 6 || P.fft_m) return nullptr;
        int m = 1;                         // automatic: parameter taps (FFMA) when one PSF (measured
                                           // 7% faster than packed FFMA2 on the 64x64 workload)
        if (want == 1) m = 0;
        if (want == 2) m = 1;
        if (want == 3) m = 2;
        if (want == 7) m = 3;
        if (m > 0 && (n_used > 1 || P.K * P.K > MAX_PTAP)) m = 0;
        const void* f = pick_fast<T>(ctx, P, m);
        if (!f && m == 1 && want == 0) {  // FFMA parameter taps are compiled for K = 9 only
            m = 2;
            f = pick_fast<T>(ctx, P, 2);
        }
        if (!f && m > 0) {
            m = 0;
            f = pick_fast<T>(ctx, P, 0);
        }
        if (f) {
            fast = true;
            mode = m;
        }
        return f;
    };
    // chained calls: each CTA slot's share of the estimated cost of the call
    double chain_budget = 0.0;
    if (lam_start) {
        double tw = 0.0;
        for (int c = 0; c < n_cand; ++c) {
            const Prob<T>& P = hp[prob_idx[c]];
            const double work = (double)P.plen * P.K * P.K + 8.0 * P.nrays;
            for (int k = 0; k < n_lam[c]; ++k) tw += work * chain_weight(n_lam[c], k);
        }
        chain_budget = tw / (double)cgls_slots(ctx, 2);
    }
    for (int c = 0; c < n_cand; ++c) {
        const Prob<T>& P = hp[prob_idx[c]];
        const int place = pick_place<T>(ctx, P, o.place);
        const bool big = place != PLACE_SMEM;
        const void* fn = pick_cgls(prec, place, P.fft_m ? 0 : P.K);
        size_t item_smem = smem_bytes<T>(P, layout_of(place));
        long long item_slab = (long long)slab_bytes<T>(P, layout_of(place));
        int per_sm = two_per_sm(place) ? 2 : 1, mode = 0;
        bool fast = false;
        if (const void* ff = choose(P, mode, fast)) {
            fn = ff;
            item_smem = fast_smem_bytes(*reinterpret_cast<const Prob<float>*>(&P));
            item_slab = (long long)fast_slab_bytes(*reinterpret_cast<const Prob<float>*>(&P));
            per_sm = 2;
        }
        if (!fn) {
            set_error("no kernel for this PSF size");
            return MIRAGE_ERR_UNSUPPORTED;
        }
        auto key = std::make_pair(fn, (int)big);
        Group& g = groups[key];
        g.fn = fn;
        g.big = big;
        g.fast = fast;
        g.prob = (g.prob == -1 || g.prob == prob_idx[c]) ? prob_idx[c] : -2;
        g.per_sm = per_sm;
        g.smem = std::max(g.smem, item_smem);
        g.slab = std::max<long long>(g.slab, item_slab);
        const double work = (double)P.plen * P.K * P.K + 8.0 * P.nrays;
        // lambda grids ascend: smaller k = smaller lambda = more CG iterations
        auto cost_of = [&](int k) { return work * (double)(n_lam[c] - k + 4); };
        if (lam_start) {
            // chains from the predicted corner: down to the smallest lambda,
            // and up from the next one.  A chain is cut into segments (each
            // further segment starts cold) whose estimated cost stays within
            // one CTA slot's share of the whole call, so that no work unit
            // outlasts the persistent queue's balance.  Costs follow the
            // iteration counts of log-spaced grids, which grow geometrically
            // towards small lambda
            const int ks = std::min(std::max(lam_start[c], 0), n_lam[c] - 1);
            auto wk = [&](int k) { return work * chain_weight(n_lam[c], k); };
            auto push_run = [&](int ka, int kb, double cd) {
                g.items.push_back({-cd, pack_chain(c, ka, kb)});
                g.cost += cd;
            };
            int ka = ks;
            double cd = 0.0;
            for (int k = ks; k >= 0; --k) {
                if (k < ka && cd + wk(k) > chain_budget) {
                    push_run(ka, k + 1, cd);
                    ka = k;
                    cd = 0.0;
                }
                cd += wk(k);
            }
            push_run(ka, 0, cd);
            if (ks + 1 < n_lam[c]) {
                ka = ks + 1;
                cd = 0.0;
                for (int k = ks + 1; k < n_lam[c]; ++k) {
                    if (k > ka && cd + wk(k) > chain_budget) {
                        push_run(ka, k - 1, cd);
                        ka = k;
                        cd = 0.0;
                    }
                    cd += wk(k);
                }
                push_run(ka, n_lam[c] - 1, cd);
            }
        } else {
            for (int k = 0; k < n_lam[c]; ++k) {
                g.items.push_back({-cost_of(k), pack_chain(c, k, k)});
                g.cost += cost_of(k);
            }
        }
    }
    std::vector<int> all_items;
    std::vector<size_t> g_off;
    std::vector<Group*> glist;
    for (auto& kv : groups) glist.push_back(&kv.second);
    // costliest group first: the others fill in behind its tail
    std::stable_sort(glist.begin(), glist.end(), [](const Group* a, const Group* b) { return a->cost > b->cost; });
    for (Group* gp : glist) {
        Group& g = *gp;
        std::stable_sort(g.items.begin(), g.items.end(),
                         [](const std::pair<double, int>& a, const std::pair<double, int>& b) { return a.first < b.first; });
        g_off.push_back(all_items.size());
        for (auto& it : g.items) all_items.push_back(it.second);
    }
    // plain mode: one candidate per launch sequence, items grouped per candidate
    std::vector<int> plain_items;
    std::vector<int> plain_off(n_cand + 1, 0);
    if (o.mode == MIRAGE_MODE_PLAIN) {
        for (int c = 0; c < n_cand; ++c) {
            plain_off[c] = (int)plain_items.size();
            for (int k = n_lam[c] - 1 + 0; k >= 0; --k) plain_items.push_back(pack_chain(c, k, k));
        }
        plain_off[n_cand] = (int)plain_items.size();
    }
    const std::vector<int>& items_v = o.mode == MIRAGE_MODE_PLAIN ? plain_items : all_items;

    const size_t n_counters = std::max<size_t>(glist.size(), (size_t)n_cand) + 1;
    // device metadata block: cand_prob[n_cand] | n_lam[n_cand] | items[...]
    std::vector<int> meta;
    meta.reserve(2 * n_cand + items_v.size());
    meta.insert(meta.end(), prob_idx, prob_idx + n_cand);
    meta.insert(meta.end(), n_lam, n_lam + n_cand);
    meta.insert(meta.end(), items_v.begin(), items_v.end());
    TRY(ctx->counters.ensure(sizeof(int) * n_counters));
    // taps of the fast kernels' launch groups (kernel parameters)
    std::vector<std::vector<float>> gtaps(glist.size());
    for (size_t gi = 0; gi < glist.size(); ++gi) {
        Group* g = glist[gi];
        if (!g->fast || g->prob < 0) continue;
        const Prob<T>& P = hp[g->prob];
        const int K = P.K;
        std::vector<T> psf((size_t)K * K);
        CK(cudaMemcpy(psf.data(), P.psf, sizeof(T) * K * K, cudaMemcpyDefault));
        std::vector<float>& tp = gtaps[gi];
        tp.assign(2 * MAX_PTAP, 0.f);
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                tp[a * K + b] = tap_value((float)psf[(K - 1 - a) * K + (K - 1 - b)], o.variant == 7);
                tp[MAX_PTAP + a * K + b] = tap_value((float)psf[a * K + b], o.variant == 7);
            }
    }
    // per-CTA global slab (bytes): FP64 refinement buffers, plus all work
    // buffers for items that do not fit in shared memory
    long long slab_stride = 0;
    std::vector<long long> g_slab_off(glist.size(), 0);  // first slab slot of each group
    long long slab_slots = 0;
    for (size_t gi = 0; gi < glist.size(); ++gi) {
        Group* g = glist[gi];
        slab_stride = std::max(slab_stride, (g->slab + 255) / 256 * 256);
        // groups run concurrently: each owns its own CTA slots of the slab
        g_slab_off[gi] = slab_slots;
        slab_slots += std::min<long long>(cgls_slots(ctx, g->per_sm), (long long)g->items.size());
    }
    if (o.mode == MIRAGE_MODE_PLAIN) slab_slots = std::max<long long>(slab_slots, max_lam);
    TRY(ctx->slab.ensure((size_t)slab_stride * std::max<long long>(slab_slots, 1)));
    if (spec_stride) TRY(ctx->spec.ensure((sizeof(double2) + sizeof(float2)) * (size_t)spec_stride * n_probs));

    // graph key: everything that shapes the launch sequence
    std::string key;
    const bool graph = o.use_graph && o.mode == MIRAGE_MODE_BATCHED;
    if (graph) {
        // a grown scratch buffer invalidates every captured graph
        std::vector<void*> now = {ctx->E.p, ctx->E64.p, ctx->Etmp.p, ctx->inv.p, ctx->cst.p, ctx->swp.p, ctx->dpad.p,
                                  ctx->nent.p, ctx->cstat.p, ctx->X.p, ctx->istat.p, ctx->slab.p, ctx->counters.p,
                                  ctx->spec.p};
        if (now != ctx->scratch_seen) {
            drop_graphs(ctx);
            ctx->scratch_seen = now;
        }
        auto addb = [&](const void* p, size_t n) { key.append(reinterpret_cast<const char*>(p), n); };
        addb(&n_cand, sizeof(n_cand));
        addb(&max_lam, sizeof(max_lam));
        addb(hp.data(), sizeof(Prob<T>) * hp.size());
        addb(meta.data(), sizeof(int) * meta.size());
        const void* ptrs[] = {d_lens, d_lambdas, d_warm, d_chi2, d_reg, d_relres, d_kappa, d_iters, d_istat,
                              d_corner, d_status, d_sout, d_allx, st};
        addb(ptrs, sizeof(ptrs));
        addb(&o.tol, sizeof(o.tol));
        addb(&o.maxit, sizeof(o.maxit));
        addb(&o.replace_every, sizeof(o.replace_every));
        addb(&o.variant, sizeof(o.variant));
        addb(&o.inner_eta, sizeof(o.inner_eta));
        addb(&o.place, sizeof(o.place));
        for (auto& tp : gtaps)
            if (!tp.empty()) addb(tp.data(), sizeof(float) * tp.size());
        auto it = ctx->graphs.find(key);
        if (it != ctx->graphs.end()) {
            CK(cudaGraphLaunch(it->second.exec, st));
            ctx->last_launches = it->second.launches;
            return MIRAGE_OK;
        }
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    }
    GraphEntry ge;
    DevBuf& probs_buf = graph ? ge.probs : ctx->probs;
    DevBuf& meta_buf = graph ? ge.meta : ctx->items;
    TRY(probs_buf.ensure(sizeof(Prob<T>) * n_probs));
    TRY(meta_buf.ensure(sizeof(int) * meta.size()));

    // uploads (before any capture)
    TRY(upload(ctx, st, {{probs_buf.p, hp.data(), sizeof(Prob<T>) * n_probs},
                         {meta_buf.p, meta.data(), sizeof(int) * meta.size()}}));

    CandScratch<T> cs;
    fill_scratch<T>(cs, ctx, false, sE, sInv, sCst, sPad);
    const Prob<T>* dprobs = probs_buf.as<Prob<T>>();
    const int* dcand = meta_buf.as<int>();
    const int* dnlam = dcand + n_cand;
    const int* ditems = dcand + 2 * n_cand;
    int* dcnt = ctx->counters.as<int>();
    const KernelTable& tb = table();

    for (Group* g : glist) TRY(set_smem(ctx, g->fn, g->smem));
    if (spec_stride) TRY(set_smem(ctx, tb.psf_spectra[prec], fft_smem_bytes(1024)));
    TRY(set_smem(ctx, tb.raytrace[prec], (size_t)max_cells * 4));
    TRY(set_smem(ctx, tb.rt_place[prec], (size_t)max_cells * 4));

    CglsArgs<T> A;
    std::memset(&A, 0, sizeof(A));
    A.probs = dprobs;
    A.cand_prob = dcand;
    A.lens = d_lens;
    A.lambdas = d_lambdas;
    A.tol = o.tol;
    A.eta = o.inner_eta > 0.0 ? o.inner_eta : 0.01;
    A.maxit = o.maxit;
    A.replace_every = o.replace_every;
    A.max_lam = max_lam;
    A.max_ns = (int)max_ns;
    A.warm_x = d_warm;
    A.cs = cs;
    A.slab = ctx->slab.p;
    A.slab_stride = slab_stride;
    A.X = dX;
    A.chi2 = d_chi2;
    A.reg = d_reg;
    A.iters = d_iters;
    A.relres = d_relres;
    A.istat = dIst;
    A.phase_clk = nullptr;
    double2* d_spec64 = nullptr;
    float2* d_spec32 = nullptr;
    if (spec_stride) {
        d_spec64 = ctx->spec.as<double2>();
        if (sizeof(T) == 4) d_spec32 = reinterpret_cast<float2*>(d_spec64 + spec_stride * n_probs);
        A.spec64 = d_spec64;
        A.spec32 = d_spec32;
        A.spec_stride = spec_stride;
    }
    if (!graph && o.threads == -2) {
        TRY(ctx->clk.ensure(FAST_NPH * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(ctx->clk.p, 0, FAST_NPH * sizeof(unsigned long long), st));
        A.phase_clk = ctx->clk.as<unsigned long long>();
    }

    const cudaStream_t launch_st = st;
    if (graph) {
        st = ctx->cap_stream;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    }
    int rc = MIRAGE_OK;
    if (spec_stride) {  // PSF spectra of the FFT problems (once per call)
        void* sa[] = {(void*)&dprobs, (void*)&d_spec64, (void*)&d_spec32, (void*)&spec_stride};
        rc = launch(ctx, tb.psf_spectra[prec], dim3(n_probs), dim3(NTHREADS), sa, fft_smem_bytes(1024), st);
    }
    do {
        if (rc) break;
        const bool timing = !graph && o.threads < 0;
        ctx->timed = 0;
        if (timing && !ctx->ev[0])
            for (int e = 0; e < 4; ++e) cudaEventCreate(&ctx->ev[e]);
        if (o.mode == MIRAGE_MODE_BATCHED) {
            if (timing) cudaEventRecord(ctx->ev[0], st);
            // 1) ray trace every candidate
            rc = launch_raytrace<T>(ctx, dprobs, dcand, d_lens, 0, n_cand, cs, max_cells, max_npix, st);
            if (rc) break;
            // 2) CGLS items, one persistent launch per kernel class
            if (cudaMemsetAsync(dcnt, 0, sizeof(int) * n_counters, st) != cudaSuccess) {
                set_error("cudaMemsetAsync failed");
                rc = MIRAGE_ERR_CUDA;
                break;
            }
            if (timing) cudaEventRecord(ctx->ev[1], st);
            // kernel groups (different kernels or placements) run on side
            // streams so that one group's tail overlaps the next group
            const bool fork = glist.size() > 1;
            if (fork) {
                if (!ctx->fork_ev) {
                    if (cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
                        set_error("cudaEventCreate failed");
                        rc = MIRAGE_ERR_CUDA;
                        break;
                    }
                    for (int i = 0; i < 4; ++i) {
                        cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking);
                        cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming);
                    }
                }
                cudaEventRecord(ctx->fork_ev, st);
                for (int i = 0; i < 4; ++i) cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0);
            }
            for (size_t gi = 0; gi < glist.size() && !rc; ++gi) {
                Group* g = glist[gi];
                const cudaStream_t gs = fork ? ctx->side[gi % 4] : st;
                A.slab = ctx->slab.as<unsigned char>() + g_slab_off[gi] * slab_stride;
                A.items = ditems + g_off[gi];
                A.n_items = (int)g->items.size();
                A.counter = dcnt + gi;
                const int grid = (int)std::min<long long>(cgls_slots(ctx, g->per_sm), (long long)g->items.size());
                if (g->fast) {
                    FastArgs fa;
                    std::memset(&fa, 0, sizeof(fa));
                    set_fast_args<T>(fa, A);
                    if (!gtaps[gi].empty()) std::memcpy(fa.ptap, gtaps[gi].data(), sizeof(fa.ptap));
                    void* args[] = {&fa};
                    rc = launch(ctx, g->fn, dim3(grid), dim3(NTHREADS), args, g->smem, gs);
                } else {
                    void* args[] = {&A};
                    rc = launch(ctx, g->fn, dim3(grid), dim3(NTHREADS), args, g->smem, gs);
                }
            }
            if (fork) {
                for (int i = 0; i < 4; ++i) {
                    cudaEventRecord(ctx->join_ev[i], ctx->side[i]);
                    cudaStreamWaitEvent(st, ctx->join_ev[i], 0);
                }
            }
            if (rc) break;
            if (timing) cudaEventRecord(ctx->ev[2], st);
            // 3) L-curve corner, status, s_out
            {
                int nc = n_cand, ml = max_lam, mns = (int)max_ns, c0 = 0;
                const int* ist = dIst;
                const int* cst = cs.cstat;
                const T* Xc = dX;
                void* args[] = {&c0, &nc, &ml, &mns, (void*)&dnlam, (void*)&dcand, (void*)&dprobs, (void*)&d_chi2,
                                (void*)&d_reg, (void*)&ist, (void*)&cst, (void*)&Xc, &d_corner, &d_kappa, &d_sout,
                                &d_status};
                rc = launch(ctx, tb.finalize[prec], dim3(n_cand), dim3(128), args, 0, st);
            }
            if (timing) {
                cudaEventRecord(ctx->ev[3], st);
                ctx->timed = 1;
            }
        } else {
            // plain: per candidate, ray trace (1 CTA), its lambdas (1 CTA each), finalize
            if (cudaMemsetAsync(dcnt, 0, sizeof(int) * n_counters, st) != cudaSuccess) {
                set_error("cudaMemsetAsync failed");
                rc = MIRAGE_ERR_CUDA;
                break;
            }
            for (int c = 0; c < n_cand && !rc; ++c) {
                const Prob<T>& P = hp[prob_idx[c]];
                const int place = pick_place<T>(ctx, P, o.place);
                const void* fn = pick_cgls(prec, place, P.fft_m ? 0 : P.K);
                size_t item_smem = smem_bytes<T>(P, layout_of(place));
                int pmode = 0;
                bool pfast = false;
                if (const void* ff = choose(P, pmode, pfast)) {
                    fn = ff;
                    item_smem = fast_smem_bytes(*reinterpret_cast<const Prob<float>*>(&P));
                }
                TRY(set_smem(ctx, fn, item_smem));
                int cand0 = c, nc = 1;
                rc = launch_raytrace<T>(ctx, dprobs, dcand, d_lens, c, 1, cs, max_cells, max_npix, st);
                if (rc) break;
                A.items = ditems + plain_off[c];
                A.n_items = plain_off[c + 1] - plain_off[c];
                A.counter = dcnt + c;
                if (pfast) {
                    FastArgs fa;
                    std::memset(&fa, 0, sizeof(fa));
                    set_fast_args<T>(fa, A);
                    if (pmode > 0) {
                        std::vector<T> psf((size_t)P.K * P.K);
                        CK(cudaMemcpy(psf.data(), P.psf, sizeof(T) * P.K * P.K, cudaMemcpyDefault));
                        for (int a = 0; a < P.K; ++a)
                            for (int b = 0; b < P.K; ++b) {
                                fa.ptap[0][a * P.K + b] =
                                    tap_value((float)psf[(P.K - 1 - a) * P.K + (P.K - 1 - b)], pmode == 3);
                                fa.ptap[1][a * P.K + b] = tap_value((float)psf[a * P.K + b], pmode == 3);
                            }
                    }
                    void* a2[] = {&fa};
                    rc = launch(ctx, fn, dim3(A.n_items), dim3(NTHREADS), a2, item_smem, st);
                } else {
                    void* a2[] = {&A};
                    rc = launch(ctx, fn, dim3(A.n_items), dim3(NTHREADS), a2, item_smem, st);
                }
                if (rc) break;
                int ml = max_lam, mns = (int)max_ns;
                const int* ist = dIst;
                const int* cst = cs.cstat;
                const T* Xc = dX;
                void* a3[] = {&cand0, &nc, &ml, &mns, (void*)&dnlam, (void*)&dcand, (void*)&dprobs, (void*)&d_chi2,
                              (void*)&d_reg, (void*)&ist, (void*)&cst, (void*)&Xc, &d_corner, &d_kappa, &d_sout,
                              &d_status};
                rc = launch(ctx, tb.finalize[prec], dim3(1), dim3(128), a3, 0, st);
            }
        }
    } while (0);

    if (graph) {
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &gr);
        if (rc != MIRAGE_OK) {
            if (gr) cudaGraphDestroy(gr);
            ge.probs.release();
            ge.meta.release();
            return rc;
        }
        if (e != cudaSuccess) {
            set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
            if (gr) cudaGraphDestroy(gr);
            return MIRAGE_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&ge.exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
            ge.probs.release();
            ge.meta.release();
            return MIRAGE_ERR_CUDA;
        }
        ge.launches = ctx->last_launches;
        GraphEntry& slot = ctx->graphs[key];
        slot = ge;
        ge.probs.p = nullptr;  // ownership moved to the cache entry
        ge.meta.p = nullptr;
        CK(cudaGraphLaunch(slot.exec, launch_st));
    }
    return rc;
}

template <typename T>
int forward_impl(mirage_ctx* ctx, const mirage_problem_t* prob, const double* lens, const void* s, int n_src,
                 void* model, double* chi2, int* status, cudaStream_t st) {
    constexpr int prec = prec_of<T>();
    ctx->last_launches = 0;
    if (!prob || !lens || !s || !chi2 || n_src < 0) {
        set_error("forward: null pointer");
        return MIRAGE_ERR_ARG;
    }
    if (check_geom(prob->geom) != MIRAGE_OK || !prob->d || !prob->sigma || !prob->mask || !prob->psf) {
        set_error("forward: bad problem");
        return MIRAGE_ERR_ARG;
    }
    if (n_src == 0) return MIRAGE_OK;
    Prob<T> P = make_prob<T>(*prob, prob->d, prob->sigma, prob->mask, prob->psf);
    if ((long long)P.ncells * 4 > ctx->max_smem - 2048) {
        set_error("source grid too large for the ray-trace kernel");
        return MIRAGE_ERR_UNSUPPORTED;
    }
    const long long sE = P.nrays, sInv = P.nrays, sCst = (P.ncells + 1 + 3) / 4 * 4, sPad = (P.plen + 3) / 4 * 4;
    TRY(ctx->fE.ensure(sizeof(Entry<T>) * sE));
    if (sizeof(T) == 4) TRY(ctx->fE64.ensure(sizeof(Entry<double>) * sE));
    TRY(ctx->fEtmp.ensure(sizeof(Entry<double>) * sE));
    TRY(ctx->finv.ensure(sizeof(int) * sInv));
    TRY(ctx->fcst.ensure(sizeof(int) * sCst));
    TRY(ctx->fswp.ensure(sizeof(T) * sPad));
    TRY(ctx->fdpad.ensure(sizeof(T) * sPad));
    TRY(ctx->fnent.ensure(sizeof(int)));
    TRY(ctx->fcstat.ensure(sizeof(int)));
    TRY(ctx->fprob.ensure(sizeof(Prob<T>) + sizeof(int)));
    const int grid = std::min(n_src, 2 * ctx->sm_count);
    const long long stride = (P.plen + 63) / 64 * 64;
    TRY(ctx->fslab.ensure(sizeof(T) * stride * grid));
    std::vector<char> up(sizeof(Prob<T>) + sizeof(int), 0);
    std::memcpy(up.data(), &P, sizeof(P));
    TRY(upload(ctx, st, {{ctx->fprob.p, up.data(), up.size()}}));
    const Prob<T>* dprob = ctx->fprob.as<Prob<T>>();
    const int* dcand = reinterpret_cast<const int*>(ctx->fprob.as<char>() + sizeof(Prob<T>));
    CandScratch<T> cs;
    fill_scratch<T>(cs, ctx, true, sE, sInv, sCst, sPad);
    const KernelTable& tb = table();
    TRY(launch_raytrace<T>(ctx, dprob, dcand, lens, 0, 1, cs, P.ncells, (long long)P.npix, st));
    if constexpr (sizeof(T) == 4) {
        // banded kernel: taps as kernel parameters, L s gathered into shared memory
        const void* fb = (P.Np == 1 && P.interp != MIRAGE_INTERP_BICUBIC && P.K < MAX_K && P.K * P.K <= MAX_FTAP)
                             ? tb.fwdb[P.K]
                             : nullptr;
        if (fb && P.tiles_x <= FWD_THREADS) {
            const int bt = std::min(FWD_THREADS / P.tiles_x, P.tiles_y);
            const size_t smb = fwd_band_smem(P, bt);
            if ((long long)smb <= ctx->max_smem) {
                TRY(ctx->fpix.ensure(sizeof(float4) * (size_t)P.npix));
                float4* pm = ctx->fpix.as<float4>();
                {
                    CandScratch<float> csv = cs;
                    const Prob<float>* dp0 = dprob;
                    void* ap[] = {(void*)&dp0, &csv, (void*)&pm};
                    TRY(launch(ctx, tb.pixmap, dim3(std::min((P.npix + NTHREADS - 1) / NTHREADS, 4 * ctx->sm_count)),
                               dim3(NTHREADS), ap, 0, st));
                }
                std::vector<unsigned char> fab(sizeof(FwdArgs), 0);
                FwdArgs* fa = reinterpret_cast<FwdArgs*>(fab.data());
                fa->probs = dprob;
                fa->cs = cs;
                fa->pixmap = pm;
                fa->S = reinterpret_cast<const float*>(s);
                fa->n_src = n_src;
                fa->model = reinterpret_cast<float*>(model);
                fa->chi2 = chi2;
                fa->status = status;
                fa->band_tiles = bt;
                TRY(set_smem(ctx, fb, smb));
                void* a3[] = {fa};
                TRY(launch(ctx, fb, dim3(std::min(n_src, ctx->sm_count)), dim3(FWD_THREADS), a3, smb, st));
                return MIRAGE_OK;
            }
        }
    }
    const void* fn = pick_fwd(prec, P.K);
    const size_t smem = align_up<T>(sizeof(T) * P.K * P.kp, 16) + 2 * 33 * sizeof(double) + 16;
    TRY(set_smem(ctx, fn, smem));
    const T* S = reinterpret_cast<const T*>(s);
    T* M = reinterpret_cast<T*>(model);
    T* slab = ctx->fslab.as<T>();
    long long sstr = stride;
    void* a2[] = {(void*)&dprob, &cs, (void*)&S, &n_src, &M, &chi2, &slab, &sstr, &status};
    TRY(launch(ctx, fn, dim3(grid), dim3(NTHREADS), a2, smem, st));
    return MIRAGE_OK;
}

// fixed-iteration CGLS with the iteration L-curve (mirage_eval_iter)
template <typename T>
int iter_impl(mirage_ctx* ctx, const mirage_problem_t* probs, int n_probs, const double* lens, const int* prob_idx,
              int n_cand, int n_iter, const void* bhat, long long bhat_stride, double* chi2, double* reg,
              double* dof, int* corner, double* kappa, void* s_out, int* status, cudaStream_t st) {
    constexpr int prec = prec_of<T>();
    ctx->last_launches = 0;
    if (n_cand == 0) return MIRAGE_OK;
    if (!probs || n_probs < 1 || !lens || !prob_idx || !chi2 || !reg || !corner || !status || n_cand < 0 ||
        n_iter < 1 || n_iter > MAX_LAM - 1 || (bhat && bhat_stride < 1)) {
        set_error("eval_iter: null pointer or size out of range (1 <= n_iter <= %d)", MAX_LAM - 1);
        return MIRAGE_ERR_ARG;
    }
    std::vector<Prob<T>> hp(n_probs);
    long long max_rays = 0, max_cells = 0, max_plen = 0, max_ns = 0, max_npix = 0;
    size_t smem = 0, slab = 0;
    int k_all = -1;
    for (int p = 0; p < n_probs; ++p) {
        if (check_geom(probs[p].geom) != MIRAGE_OK || !probs[p].d || !probs[p].sigma || !probs[p].mask ||
            !probs[p].psf) {
            set_error("eval_iter: bad problem %d", p);
            return MIRAGE_ERR_ARG;
        }
        hp[p] = make_prob<T>(probs[p], probs[p].d, probs[p].sigma, probs[p].mask, probs[p].psf);
        if (bhat && (long long)probs[p].geom.nx * probs[p].geom.ny > bhat_stride) {
            set_error("eval_iter: bhat_stride below the pixel count of problem %d", p);
            return MIRAGE_ERR_ARG;
        }
        max_rays = std::max<long long>(max_rays, hp[p].nrays);
        max_cells = std::max<long long>(max_cells, hp[p].ncells);
        max_plen = std::max<long long>(max_plen, hp[p].plen);
        max_ns = std::max<long long>(max_ns, hp[p].ns);
        max_npix = std::max<long long>(max_npix, hp[p].npix);
        smem = std::max(smem, iter_smem_bytes<T>(hp[p].K, hp[p].kp));
        slab = std::max(slab, iter_slab_bytes<T>(hp[p], n_iter));
        k_all = (k_all == -1 || k_all == hp[p].K) ? hp[p].K : 0;
    }
    for (int c = 0; c < n_cand; ++c)
        if (prob_idx[c] < 0 || prob_idx[c] >= n_probs) {
            set_error("eval_iter: bad prob_idx of candidate %d", c);
            return MIRAGE_ERR_ARG;
        }
    if (max_cells * 4 > ctx->max_smem - 2048) {
        set_error("source grid too large for the ray-trace kernel");
        return MIRAGE_ERR_UNSUPPORTED;
    }
    const long long sE = max_rays, sInv = max_rays, sCst = (max_cells + 1 + 3) / 4 * 4, sPad = (max_plen + 3) / 4 * 4;
    TRY(ctx->E.ensure(sizeof(Entry<T>) * n_cand * sE));
    if (sizeof(T) == 4) TRY(ctx->E64.ensure(sizeof(Entry<double>) * n_cand * sE));
    TRY(ctx->Etmp.ensure(sizeof(Entry<double>) * n_cand * sE));
    TRY(ctx->inv.ensure(sizeof(int) * n_cand * sInv));
    TRY(ctx->cst.ensure(sizeof(int) * n_cand * sCst));
    TRY(ctx->swp.ensure(sizeof(T) * n_cand * sPad));
    TRY(ctx->dpad.ensure(sizeof(T) * n_cand * sPad));
    TRY(ctx->nent.ensure(sizeof(int) * n_cand));
    TRY(ctx->cstat.ensure(sizeof(int) * n_cand));
    TRY(ctx->probs.ensure(sizeof(Prob<T>) * n_probs));
    TRY(ctx->cand_prob.ensure(sizeof(int) * n_cand));
    TRY(ctx->counters.ensure(sizeof(int)));
    const int grid = std::min(n_cand, 2 * ctx->sm_count);
    TRY(ctx->slab.ensure(slab * grid));
    TRY(upload(ctx, st, {{ctx->probs.p, hp.data(), sizeof(Prob<T>) * n_probs},
                         {ctx->cand_prob.p, prob_idx, sizeof(int) * n_cand}}));
    CK(cudaMemsetAsync(ctx->counters.p, 0, sizeof(int), st));
    CandScratch<T> cs;
    fill_scratch<T>(cs, ctx, false, sE, sInv, sCst, sPad);
    const Prob<T>* dprobs = ctx->probs.as<Prob<T>>();
    const int* dcand = ctx->cand_prob.as<int>();
    const KernelTable& tb = table();
    TRY(launch_raytrace<T>(ctx, dprobs, dcand, lens, 0, n_cand, cs, max_cells, max_npix, st));
    const void* fn = (k_all > 0 && k_all < MAX_K && tb.iter[prec][k_all]) ? tb.iter[prec][k_all] : tb.iter[prec][0];
    TRY(set_smem(ctx, fn, smem));
    IterArgs<T> A;
    std::memset(&A, 0, sizeof(A));
    A.probs = dprobs;
    A.cand_prob = dcand;
    A.cs = cs;
    A.n_cand = n_cand;
    A.n_iter = n_iter;
    A.max_ns = (int)max_ns;
    A.bhat = reinterpret_cast<const T*>(bhat);
    A.bhat_stride = bhat_stride;
    A.counter = ctx->counters.as<int>();
    A.slab = ctx->slab.p;
    A.slab_stride = (long long)slab;
    A.chi2 = chi2;
    A.reg = reg;
    A.dof = dof;
    A.kappa = kappa;
    A.corner = corner;
    A.s_out = reinterpret_cast<T*>(s_out);
    A.status = status;
    void* a2[] = {&A};
    TRY(launch(ctx, fn, dim3(grid), dim3(NTHREADS), a2, smem, st));
    return MIRAGE_OK;
}

}  // namespace

extern "C" {

int mirage_create(mirage_ctx_t** out, int device, int precision) {
    if (!out) return MIRAGE_ERR_ARG;
    *out = nullptr;
    if (precision != MIRAGE_FP32 && precision != MIRAGE_FP64) {
        set_error("precision must be MIRAGE_FP32 or MIRAGE_FP64");
        return MIRAGE_ERR_ARG;
    }
    CK(cudaSetDevice(device));
    mirage_ctx* c = new mirage_ctx();
    c->device = device;
    c->precision = precision;
    cudaError_t e1 = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e2 = cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaError_t e3 = cudaDeviceGetAttribute(&c->max_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("cudaDeviceGetAttribute failed");
        delete c;
        return MIRAGE_ERR_CUDA;
    }
    (void)table();
    *out = c;
    return MIRAGE_OK;
}

int mirage_destroy(mirage_ctx_t* ctx) {
    if (!ctx) return MIRAGE_OK;
    cudaSetDevice(ctx->device);
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (int i = 0; i < 4; ++i) {
        if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
        if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    for (int e = 0; e < 4; ++e)
        if (ctx->ev[e]) cudaEventDestroy(ctx->ev[e]);
    DevBuf* bufs[] = {&ctx->E, &ctx->E64, &ctx->Etmp, &ctx->inv, &ctx->cst, &ctx->swp, &ctx->dpad, &ctx->nent, &ctx->cstat,
                      &ctx->X, &ctx->istat, &ctx->slab, &ctx->probs, &ctx->cand_prob, &ctx->items, &ctx->counters,
                      &ctx->stage, &ctx->fE, &ctx->fE64, &ctx->fEtmp, &ctx->finv, &ctx->fcst, &ctx->fswp, &ctx->fdpad,
                      &ctx->fnent, &ctx->fcstat, &ctx->fslab, &ctx->fprob, &ctx->fcand, &ctx->fpix, &ctx->rt_cursor, &ctx->clk,
                      &ctx->spec};
    for (DevBuf* b : bufs) b->release();
    if (ctx->pin_pending) cudaEventSynchronize(ctx->pin_ev);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->pin_ev) cudaEventDestroy(ctx->pin_ev);
    delete ctx;
    return MIRAGE_OK;
}

int mirage_eval_batch(mirage_ctx_t* ctx, const mirage_problem_t* probs, int n_probs, const double* lens,
                      const int* prob_idx, int n_cand, const double* lambdas, const int* n_lam, int max_lam,
                      const mirage_opts_t* opts, const void* warm_x, const int* lam_start, double* chi2,
                      double* reg, int* iters, double* relres, int* item_status, int* corner, double* kappa,
                      void* s_out, void* all_x, int* status, void* stream) {
    if (!ctx || !opts) return MIRAGE_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return MIRAGE_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ctx->precision == MIRAGE_FP32)
        return eval_impl<float>(ctx, probs, n_probs, lens, prob_idx, n_cand, lambdas, n_lam, max_lam, opts, warm_x,
                                lam_start, chi2, reg, iters, relres, item_status, corner, kappa, s_out, all_x, status, st);
    return eval_impl<double>(ctx, probs, n_probs, lens, prob_idx, n_cand, lambdas, n_lam, max_lam, opts, warm_x,
                             lam_start, chi2, reg, iters, relres, item_status, corner, kappa, s_out, all_x, status, st);
}

int mirage_lcurve(const double* chi2, const double* reg, const int* n_lam, int n_cand, int max_lam, int* corner,
                  double* kappa, int* flags, void* stream) {
    if (n_cand == 0) return MIRAGE_OK;
    if (!chi2 || !reg || !n_lam || !corner || n_cand < 0 || max_lam < 1 || max_lam > MAX_LAM) {
        set_error("lcurve: bad argument");
        return MIRAGE_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_lcurve<0><<<(n_cand + 127) / 128, 128, 0, st>>>(chi2, reg, n_lam, n_cand, max_lam, corner, kappa, flags);
    CK(cudaGetLastError());
    return MIRAGE_OK;
}

int mirage_forward(mirage_ctx_t* ctx, const mirage_problem_t* prob, const double* lens, const void* s, int n_src,
                   void* model, double* chi2, int* status, void* stream) {
    if (!ctx) return MIRAGE_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return MIRAGE_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ctx->precision == MIRAGE_FP32) return forward_impl<float>(ctx, prob, lens, s, n_src, model, chi2, status, st);
    return forward_impl<double>(ctx, prob, lens, s, n_src, model, chi2, status, st);
}

int mirage_eval_iter(mirage_ctx_t* ctx, const mirage_problem_t* probs, int n_probs, const double* lens,
                     const int* prob_idx, int n_cand, int n_iter, const void* bhat, long long bhat_stride,
                     double* chi2, double* reg, double* dof, int* corner, double* kappa, void* s_out, int* status,
                     void* stream) {
    if (!ctx) return MIRAGE_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return MIRAGE_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ctx->precision == MIRAGE_FP32)
        return iter_impl<float>(ctx, probs, n_probs, lens, prob_idx, n_cand, n_iter, bhat, bhat_stride, chi2, reg,
                                dof, corner, kappa, s_out, status, st);
    return iter_impl<double>(ctx, probs, n_probs, lens, prob_idx, n_cand, n_iter, bhat, bhat_stride, chi2, reg, dof,
                             corner, kappa, s_out, status, st);
}

int mirage_set_reserved_slots(mirage_ctx_t* ctx, int slots) {
    if (!ctx || slots < 0) {
        set_error("set_reserved_slots: bad arguments");
        return MIRAGE_ERR_ARG;
    }
    if (slots != ctx->reserved) drop_graphs(ctx);  // captured launches carry the old grid
    ctx->reserved = slots;
    return MIRAGE_OK;
}

int mirage_last_launch_count(const mirage_ctx_t* ctx) { return ctx ? ctx->last_launches : 0; }

static_assert(MAX_LAM == MIRAGE_MAX_LAM, "lambda grid limit of the header and the kernels");

int mirage_last_phase_clocks(mirage_ctx_t* ctx, unsigned long long* clk) {
    static_assert(FAST_NPH == MIRAGE_N_PHASE_CLOCKS, "phase clock count of the header and the kernel");
    if (!ctx || !clk || !ctx->clk.p) return MIRAGE_ERR_ARG;
    CK(cudaMemcpy(clk, ctx->clk.p, FAST_NPH * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return MIRAGE_OK;
}

int mirage_last_phase_ms(mirage_ctx_t* ctx, double* ms) {
    if (!ctx || !ms) return MIRAGE_ERR_ARG;
    if (!ctx->timed) {
        set_error("no timed batched call on this context");
        return MIRAGE_ERR_ARG;
    }
    for (int i = 0; i < 3; ++i) {
        float t = 0.f;
        CK(cudaEventSynchronize(ctx->ev[i + 1]));
        CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
        ms[i] = t;
    }
    return MIRAGE_OK;
}

const char* mirage_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Internal accessors shared with the allocation-free entry point (noalloc.cu).
namespace mirage {
const KernelTable& kernel_table() { return table(); }
int geometry_ok(const mirage_geom_t& g) { return check_geom(g); }
template <typename T>
Prob<T> problem_layout(const mirage_problem_t& p) {
    return make_prob<T>(p, p.d, p.sigma, p.mask, p.psf);
}
template Prob<float> problem_layout<float>(const mirage_problem_t&);
template Prob<double> problem_layout<double>(const mirage_problem_t&);
}  // namespace mirage
