/*
 * mirage.h -- C ABI of the GB300 lens-inversion inner loop.
 *
 * For each candidate lens (SIE plus external shear) the library ray-traces
 * the image pixels to the source plane (Eq. thinlens, Eqs. SIEX/SIEY),
 * forms the bilinear lens operator L implicitly (Section 2.2), blurs with
 * the PSF B by direct zero-padded convolution (the operator the paper
 * applies by FFT, Section 2.2), and solves the regularised normal equations
 *     (L^T B^T W B L + lambda H^T H) s = L^T B^T W d        (Eqs. eqLS, TKReg)
 * with W = diag(m / sigma^2), m = mask AND mapped, by matrix-free conjugate
 * gradient for least squares (CGLS, Section 2.2 and 2.4) over a grid of
 * lambda values, then picks the L-curve corner by maximum curvature of
 * natural cubic splines in chord length (Section 2.6).  Neither L nor B is
 * ever assembled.
 *
 * Conventions shared by every entry point:
 *  - Images are row-major [ny][nx] with x the fast axis; pixel (i, j) has
 *    centre (cx + (i - (nx-1)/2) pix, cy + (j - (ny-1)/2) pix).
 *  - The source grid [sy][sx] spans the edges [sxmin, sxmax] x [symin, symax];
 *    its pixel centres lie half a cell inside.  A ray is mapped when it lies
 *    in the rectangle of the first and last source-pixel centres.
 *  - Lens vectors are 7 doubles (b, q, phi, x0, y0, gamma, theta_g): Einstein
 *    radius b >= 0, axis ratio 0 < q <= 1, major-axis angle phi (rad), lens
 *    centre, external shear gamma at angle theta_g about the lens centre.
 *  - "real" is float in MIRAGE_FP32 contexts and double in MIRAGE_FP64
 *    contexts.  FP32 contexts do the ray trace, interpolation, convolution and
 *    CG vectors in float and every inner product, norm, chi^2 and curvature
 *    in double; FP64 contexts do everything in double.
 *  - Unless a call says otherwise, array arguments are device pointers owned
 *    by the caller.  Calls are asynchronous on `stream` (a cudaStream_t, NULL
 *    = legacy default stream) unless MIRAGE_MEM_HOST is requested.
 *  - Return value: MIRAGE_OK or a negative MIRAGE_ERR_* code.  A bad
 *    candidate never fails a batch: it gets a status flag instead.
 *  - A context is not thread-safe: serialise calls that share one.
 */
#ifndef MIRAGE_H
#define MIRAGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MIRAGE_OK 0
#define MIRAGE_ERR_ARG (-1)         /* invalid argument (sizes, null pointers, geometry) */
#define MIRAGE_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define MIRAGE_ERR_NOMEM (-3)       /* device allocation of context scratch failed */
#define MIRAGE_ERR_UNSUPPORTED (-4) /* shape outside what the library supports */

#define MIRAGE_FP32 0
#define MIRAGE_FP64 1

#define MIRAGE_REG_IDENTITY 0  /* H = I (zeroth order, Section 2.1) */
#define MIRAGE_REG_GRADIENT 1  /* H = [Dx; Dy], forward differences, zero beyond the grid */
#define MIRAGE_REG_LAPLACIAN 2 /* H = 5-point Laplacian, zero beyond the grid */

/* Source-plane interpolation of a traced ray (Section 2.1): bilinear over the
 * four centres of its cell (TK04); all its weight on the nearest centre
 * (WD03's ray shooting; a tie at mid-cell goes to the upper centre); or
 * bicubic over the 4 x 4 centres around its cell with Keys' cubic-convolution
 * kernel (a = -1/2), centres beyond the grid holding no source.  A ray is
 * mapped iff it lies within the rectangle of the first and last centres, for
 * all three.  Bicubic problems run on the general CGLS kernel and the
 * general forward kernel. */
#define MIRAGE_INTERP_BILINEAR 0
#define MIRAGE_INTERP_NEAREST 1
#define MIRAGE_INTERP_BICUBIC 2

/* per-(candidate, lambda) and per-candidate status bits */
#define MIRAGE_ST_MAXIT 1        /* CG stopped at maxit above the tolerance */
#define MIRAGE_ST_STAGNATION 2   /* CG residual stopped decreasing above the tolerance */
#define MIRAGE_ST_BREAKDOWN 4    /* p^T A p <= 0 or not finite */
#define MIRAGE_ST_BAD_PARAM 8    /* lens vector not finite, b < 0 or q outside (0, 1] */
#define MIRAGE_ST_EMPTY_MAP 16   /* no pixel is both masked in and mapped */
#define MIRAGE_ST_LCURVE_FLAT 32 /* fewer than 3 distinct L-curve points or zero curvature */

#define MIRAGE_MEM_DEVICE 0 /* all arrays of the call are device memory */
#define MIRAGE_MEM_HOST 1   /* all arrays of the call are host memory; the call
                               stages them and returns after the results are back */

#define MIRAGE_MODE_BATCHED 0 /* all (candidate, lambda) items in persistent launches */
#define MIRAGE_MODE_PLAIN 1   /* one candidate per launch sequence, its lambdas in parallel */

typedef struct {
    int nx, ny;           /* image size in pixels (>= 1) */
    double pix;           /* pixel size (arcsec, > 0) */
    double cx, cy;        /* image centre (arcsec) */
    int sx, sy;           /* source grid size (>= 2 each) */
    double sxmin, sxmax;  /* source grid edges on x (sxmax > sxmin) */
    double symin, symax;  /* source grid edges on y */
    int kpsf;             /* PSF side, odd, 1 <= kpsf <= MIRAGE_MAX_KPSF */
    int subpix;           /* n: each pixel traced as n x n sub-pixels (1 <= n <= 8) */
    int reg;              /* MIRAGE_REG_* */
    int interp;           /* MIRAGE_INTERP_*: source-plane interpolation of each ray */
} mirage_geom_t;

typedef struct {
    mirage_geom_t geom;          /* host struct */
    const void* d;               /* [ny*nx] real: observed image */
    const void* sigma;           /* [ny*nx] real: noise sigma, > 0 where mask != 0 */
    const uint8_t* mask;         /* [ny*nx]: nonzero = pixel used in chi^2 and the solve */
    const void* psf;             /* [kpsf*kpsf] real, row-major, centre at (k-1)/2 */
} mirage_problem_t;

typedef struct {
    double tol;        /* stop when ||rhs - A s|| <= tol ||rhs||, the residual of the
                          solution evaluated in FP64 */
    int maxit;         /* CG iteration cap per (candidate, lambda), summed over the
                          refinement's inner solves; <= 0: 25 * ns */
    int mode;          /* MIRAGE_MODE_* */
    int mem;           /* MIRAGE_MEM_* */
    int use_graph;     /* 1: capture the batched launch sequence once per argument
                          set and replay it on identical calls */
    int threads;       /* 0 = default; -1 = record per-phase CUDA events on the
                          stream (non-graph batched calls) for mirage_last_phase_ms;
                          -2 = also accumulate per-phase SM clocks inside the
                          fast CGLS kernel for mirage_last_phase_clocks */
    int replace_every; /* reserved (0) */
    int variant;       /* CGLS kernel choice: 0 = automatic; 1 = two-CTA kernel with taps
                          in shared memory; 2 = two-CTA kernel with taps as kernel
                          parameters (FFMA); 3 = the same with packed FFMA2; 4 = the
                          general one-CTA kernel; 5 = the general kernel with every
                          convolution by FFT (Section 2.2); 6 = the general kernel
                          with direct convolution at any PSF width; 7 = the
                          two-CTA kernel with the inner solves' convolution
                          factors rounded to TF32 (the arithmetic of a TF32
                          tensor-core B/B^T; 9x9 PSFs, one PSF per call; an
                          experiment on the inner solves' precision, the
                          refinement's residual stays exact).  Automatic
                          choice: FFT for PSFs of 23 x 23 and wider, direct below.
                          Forced choices fall back to the general kernel where
                          they do not apply.  Other values: MIRAGE_ERR_ARG. */
    double inner_eta;  /* FP32 contexts: the relative residual reduction each inner
                          solve of the refinement aims for (each solve stops at
                          max(inner_eta, min(0.5, 0.8 tol / current residual))); 0 = the
                          default 0.01; otherwise 1e-4 <= inner_eta <= 0.5, else
                          MIRAGE_ERR_ARG.  Changes the iteration path, not the
                          solution (to tol).  FP64 contexts ignore it. */
    int place;         /* work-buffer placement of the general kernel: 0 = automatic
                          (the most on-chip placement that fits; all in the slab
                          means 4 where that kernel is compiled for the PSF width),
                          1 = all in shared
                          memory, 2 = convolution inputs and source vectors in
                          shared memory, the rest in an L2-resident slab, 3 = all in
                          the slab, 4 = all in the slab with two CTAs per SM (the
                          kernel held to 128 registers a thread; FP32 contexts,
                          else 3), 5 = as 2 with two CTAs per SM (FP32, where two
                          CTAs' shared memory fits an SM, else automatic); a
                          placement that does not fit, or a problem on
                          the FFT path (always 3), keeps the automatic one.  Other
                          values: MIRAGE_ERR_ARG. */
} mirage_opts_t;

typedef struct mirage_ctx mirage_ctx_t;

/* Create a context on CUDA device `device` with MIRAGE_FP32 or MIRAGE_FP64
 * arithmetic.  The context owns its scratch memory (grown on demand) and
 * its captured graphs; *ctx is NULL on failure. */
int mirage_create(mirage_ctx_t** ctx, int device, int precision);

/* Release every resource of the context.  NULL is accepted. */
int mirage_destroy(mirage_ctx_t* ctx);

#define MIRAGE_MAX_LAM 64 /* longest lambda grid of one candidate */
#define MIRAGE_MAX_KPSF 65 /* widest PSF (the 65 x 65 class of the paper's large test, Section 2.7) */

/* Evaluate n_cand candidate lenses (the inner loop of Section 3: ray trace,
 * CGLS on Eq. TKReg for every lambda of the candidate, L-curve corner).
 *
 *  probs[n_probs]      host array of problem descriptors (device data pointers)
 *  lens[n_cand*7]      lens vectors (double)
 *  prob_idx[n_cand]    HOST array: problem of each candidate, in [0, n_probs)
 *  lambdas[n_cand*max_lam]  lambda grid per candidate (double, > 0, ascending);
 *                      1 <= max_lam <= MIRAGE_MAX_LAM, else MIRAGE_ERR_ARG
 *  n_lam[n_cand]       HOST array: lambdas used per candidate, 1..max_lam
 *  warm_x              nullable [n_cand*max_lam*max_ns] real: CG start per
 *                      item (max_ns = the largest sx*sy of the problems);
 *                      NULL = start from zero (the paper's blank source)
 *  lam_start           nullable HOST array [n_cand]: a predicted corner index
 *                      per candidate (clamped to [0, n_lam-1]).  When given
 *                      (batched mode), each candidate's lambdas are solved as
 *                      chains: lam_start down to 0 and lam_start+1 up to
 *                      n_lam-1, each cut into segments whose estimated cost
 *                      stays within one CTA slot's share of the call; every lambda
 *                      after the first of its chain starts from the solution
 *                      of its neighbour nearer to lam_start (a chain's first
 *                      lambda starts from warm_x, or zero).  Results agree
 *                      with unchained calls to the solver tolerance.  Ignored
 *                      in plain mode.
 * Outputs ([n_cand*max_lam] unless noted; entries beyond n_lam untouched):
 *  chi2, reg           double: Eq. chi2 of the solution and ||H s||^2
 *  iters               int: CG iterations used
 *  relres              double: TRUE ||rhs - A s|| / ||rhs|| at exit (nullable)
 *  item_status         int: MIRAGE_ST_* bits per item (nullable)
 *  corner[n_cand]      int: L-curve corner index (the fitness is chi2 there)
 *  kappa               double: curvature at each knot (nullable)
 *  s_out               nullable [n_cand*max_ns] real: solution at the corner
 *  all_x               nullable [n_cand*max_lam*max_ns] real: every solution
 *  status[n_cand]      int: OR of the candidate's item bits and its own
 * With opts->mem == MIRAGE_MEM_HOST every array above (and the problem data)
 * is host memory instead, and the call blocks until the outputs are written.
 */
int mirage_eval_batch(mirage_ctx_t* ctx, const mirage_problem_t* probs, int n_probs,
                      const double* lens, const int* prob_idx, int n_cand,
                      const double* lambdas, const int* n_lam, int max_lam,
                      const mirage_opts_t* opts, const void* warm_x, const int* lam_start,
                      double* chi2, double* reg, int* iters, double* relres, int* item_status,
                      int* corner, double* kappa, void* s_out, void* all_x, int* status,
                      void* stream);

/* The paper's own inner loop (Sections 2.4-2.6): for each candidate, CGLS on
 * the weighted least-squares problem min ||sqrt(W)(B L s - d)|| from a blank
 * source (no explicit regulariser) for exactly n_iter iterations; after
 * iteration k (k = 0..n_iter, k = 0 being s = 0) it records the image chi^2
 * of s_k and the zeroth-order regularisation measure sum s_k^2, and picks the
 * corner of the L-curve (log10 sum s_k^2, log10 chi^2_k) over k = 1..n_iter
 * by the rule of mirage_lcurve.  With bhat it also runs the twin CGLS of
 * Section 2.5 on m * bhat (m = mask and mapped) with the same step
 * coefficients and records dof_k = bhat^T (bhat - A xhat_k), the Monte Carlo
 * estimate of the residual degrees of freedom (reduced chi^2 = chi^2_k /
 * dof_k).  Device memory; asynchronous on `stream` after a short host sync of
 * the uploads.
 *  probs, n_probs, lens, prob_idx (HOST), n_cand: as for mirage_eval_batch
 *  n_iter        1 .. MIRAGE_MAX_LAM-1 (the paper uses 40)
 *  bhat          nullable [n_probs*bhat_stride] real: one standard-normal
 *                image per problem, row-major (y slow), bhat_stride >= nx*ny
 *  chi2, reg     [n_cand*(n_iter+1)] double
 *  dof           nullable [n_cand*(n_iter+1)] double (needs bhat)
 *  corner        [n_cand] int: the corner iteration (1..n_iter)
 *  kappa         nullable [n_cand*(n_iter+1)] double: curvature at each k
 *  s_out         nullable [n_cand*max_ns] real: s at the corner iteration
 *  status        [n_cand] int: MIRAGE_ST_* bits (BREAKDOWN when a step
 *                coefficient is not finite; LCURVE_FLAT)
 * The iteration is unpreconditioned by design: the iteration count is the
 * regulariser, and a preconditioner would change which solution it selects. */
int mirage_eval_iter(mirage_ctx_t* ctx, const mirage_problem_t* probs, int n_probs,
                     const double* lens, const int* prob_idx, int n_cand, int n_iter,
                     const void* bhat, long long bhat_stride,
                     double* chi2, double* reg, double* dof, int* corner, double* kappa,
                     void* s_out, int* status, void* stream);

/* L-curve corner (Section 2.6) for n_cand curves of n_lam[c] points each:
 * points (log10 reg, log10 chi2) in lambda order, chord-length parameter,
 * natural cubic splines, curvature |x'y'' - y'x''| / (x'^2 + y'^2)^1.5 at
 * the knots, argmax (ties to the smaller index).  Points within 1e-12 of
 * the total chord length of their predecessor are merged (kappa 0); with
 * fewer than 3 distinct points or kappa * chord length <= 1e-9 everywhere
 * the middle index is returned with MIRAGE_ST_LCURVE_FLAT.
 *  chi2, reg [n_cand*max_lam] double, n_lam [n_cand] int (all device)
 *  corner [n_cand] int, kappa [n_cand*max_lam] double (nullable),
 *  flags [n_cand] int (nullable; receives MIRAGE_ST_LCURVE_FLAT or 0). */
int mirage_lcurve(const double* chi2, const double* reg, const int* n_lam, int n_cand, int max_lam,
                  int* corner, double* kappa, int* flags, void* stream);

/* Forward model and chi^2 of n_src source vectors at one lens (the forward
 * pass of Eq. mapping and Eq. chi2, used by the positivity refinement stage
 * of Section 3.2):  model_k = B L s_k,  chi2_k = sum_j m_j (model_k - d)_j^2 / sigma_j^2.
 *  prob      host descriptor (device data)
 *  lens[7]   device double
 *  s         [n_src*ns] real (device)
 *  model     nullable [n_src*npix] real (device)
 *  chi2      [n_src] double (device)
 *  status    nullable [1] int (device): MIRAGE_ST_BAD_PARAM / EMPTY_MAP bits */
int mirage_forward(mirage_ctx_t* ctx, const mirage_problem_t* prob, const double* lens,
                   const void* s, int n_src, void* model, double* chi2, int* status, void* stream);

/* Leave `slots` CTA slots of the device free in this context's CGLS
 * launches (the persistent kernels otherwise fill every SM), so that work on
 * other streams, such as surrogate training, can run beside the solves.
 * 0 (the default) uses the whole device.  The results do not depend on it. */
int mirage_set_reserved_slots(mirage_ctx_t* ctx, int slots);

/* Number of kernel launches the last eval/forward call of this context
 * issued (a replayed graph counts its kernels). */
int mirage_last_launch_count(const mirage_ctx_t* ctx);

/* Device time (ms) of the three phases of the last batched, non-graph call
 * made with opts->threads < 0: ms[0] ray trace, ms[1] CGLS items, ms[2]
 * L-curve/finalize.  Waits for those events. */
int mirage_last_phase_ms(mirage_ctx_t* ctx, double* ms);

/* Per-phase SM clock totals (thread 0 of each CTA, summed over CTAs) of the
 * last call made with opts->threads == -2 that ran the fast CGLS kernel,
 * MIRAGE_N_PHASE_CLOCKS values: [0] L p and H p, [1] B convolution, [2] its
 * reduction, [3] vector updates and residual store, [4] B^T convolution,
 * [5] L^T ray walk, [6] L^T join of cells split between walks, [7] L^T
 * gather and H^T, [8] its reduction, [9] p update, [10] FP64 refinement
 * residuals, [11] item set-up.  `clk` holds MIRAGE_N_PHASE_CLOCKS values.
 * Synchronous. */
#define MIRAGE_N_PHASE_CLOCKS 12
int mirage_last_phase_clocks(mirage_ctx_t* ctx, unsigned long long* clk);

/* Text of the last error raised on the calling thread ("" if none). */
const char* mirage_last_error(void);

/* ------------------------------------------------------------------------
 * Surrogate network (the learned screen in front of the exact solves).
 * A multilayer perceptron dims[0] -> dims[1] -> ... -> dims[n_layers]: SiLU
 * after every hidden layer, linear output, mean-squared-error loss, Adam
 * (b1 0.9, b2 0.999, eps 1e-8).  Products run on the tcgen05 tensor cores
 * (BF16 operands, FP32 accumulation in tensor memory; if a product's
 * completion wait runs out, about a second, its output tile is NaN); master
 * weights, moments and activations' gradients
 * are FP32.  Parameters are ordered W_1 [dims[1] x dims[0]] (row-major),
 * b_1 [dims[1]], W_2, b_2, ...  Device arrays unless noted; the network
 * object owns its weights and work buffers.  The paper's optimisers use no
 * surrogate; this serves the batched GA front end.
 * ------------------------------------------------------------------------ */
typedef struct mirage_mlp mirage_mlp_t;

/* New network on `device` with He-initialised weights from `seed`. */
int mirage_mlp_create(mirage_mlp_t** mlp, int device, int n_layers, const int* dims,
                      unsigned long long seed);
int mirage_mlp_destroy(mirage_mlp_t* mlp);
/* Number of parameters (weights and biases). */
long mirage_mlp_num_params(const mirage_mlp_t* mlp);
/* Copy FP32 parameters from / to HOST memory; setting resets Adam. */
int mirage_mlp_set_params(mirage_mlp_t* mlp, const float* host_params, long n);
int mirage_mlp_get_params(const mirage_mlp_t* mlp, float* host_params, long n);
/* y [n x dims[L]] = network(x [n x dims[0]]) (FP32 in and out). */
int mirage_mlp_forward(mirage_mlp_t* mlp, const float* x, int n, float* y, void* stream);
/* Gradient of mean((y - t)^2) into grad [num_params] (nullable), the loss
 * into loss [1] (double, nullable) and the forward output into y. */
int mirage_mlp_grad(mirage_mlp_t* mlp, const float* x, const float* t, int n, float* grad, double* loss,
                    float* y, void* stream);
/* One Adam step at learning rate lr on the batch (x, t). */
int mirage_mlp_train_step(mirage_mlp_t* mlp, const float* x, const float* t, int n, float lr,
                          double* loss, float* y, void* stream);
/* `steps` Adam steps at learning rate lr, each on `batch` rows drawn from
 * the dataset (x [n x dims[0]], t [n x dims[L]], device FP32) on the
 * device: step k takes row h(seed, k, j) mod n for slot j, with h a
 * counter-based hash (splitmix64), so no host round trip happens between
 * steps.  The launch sequence of one step is captured once per call as a
 * CUDA graph on a private stream and replayed `steps` times on `stream`.
 * Do not call while `stream` itself is being captured.  x and t must stay
 * valid until the work on `stream` completes. */
int mirage_mlp_train(mirage_mlp_t* mlp, const float* x, const float* t, int n, int steps, int batch,
                     float lr, unsigned long long seed, void* stream);
const char* mirage_mlp_last_error(void);

/* Allocation-free forward model.  The paper has no counterpart: this entry
 * exists for callers that must not let the library allocate device memory
 * (a host framework that owns the device-memory budget through its own
 * pool, or a loop where cudaMalloc / cudaFree would synchronise the device
 * at the wrong time).  It computes what mirage_forward computes, with the
 * same kernels, but needs no context and calls no cudaMalloc, cudaFree or
 * other allocating routine: all scratch comes from one fixed array of
 * mirage_noalloc_capacity() bytes (8 MiB) that every device loading the
 * library holds until the process exits.
 *  precision  MIRAGE_FP32 or MIRAGE_FP64 (the type of "real" below)
 *  prob, lens, s, n_src, model, chi2, status: as for mirage_forward; the
 *             call works on the current CUDA device.
 * Returns MIRAGE_ERR_UNSUPPORTED (message in mirage_noalloc_last_error)
 * when the problem needs more scratch than the array holds, roughly images
 * above 160 x 160 FP32 rays.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) once and keeps it for the
 * life of the process; make that first call before any stream capture, and
 * do not call this entry point on a device after cudaDeviceReset of it.
 * All calls share the array and it keeps the last call's contents (each
 * call rebuilds what it reads), so calls that overlap on the GPU (different
 * streams or threads on one device) race: serialise them.  The error text
 * is kept per calling thread. */
int mirage_forward_noalloc(int precision, const mirage_problem_t* prob, const double* lens,
                           const void* s, int n_src, void* model, double* chi2, int* status,
                           void* stream);

/* Error text of the last failed mirage_forward_noalloc call. */
const char* mirage_noalloc_last_error(void);

/* Size in bytes of the fixed scratch array of mirage_forward_noalloc. */
size_t mirage_noalloc_capacity(void);

/* Repeated PSF blur of a batch of images on one of two engines.  A
 * measurement entry point, not a step of the solve path: it times the blur
 * B of the linear system (Section 2.2; the paper applies it by FFT) as the
 * FP32 inner solves apply it, against a tensor-core form of it.
 *  engine  MIRAGE_BLUR_FFMA: the CG kernel's FP32 FFMA register tiles (4 x 4
 *          outputs per thread, taps as kernel parameters);
 *          MIRAGE_BLUR_TC_TF32: block-Toeplitz products on the tcgen05
 *          tensor cores (strips of 16 output columns, M = 128 stacked rows,
 *          a 24 x 16 Toeplitz matrix per PSF row), both factors rounded to
 *          TF32 (nearest), FP32 accumulation in tensor memory.
 *  img     device, n images of ny x nx FP32, row-major, back to back;
 *          16-byte aligned
 *  out     device, same layout (may not alias img): B applied `reps` times
 *          to each image, (B x)(y, x) = sum_ij psf(i, j) x(y - i + h,
 *          x - j + h) with h = (K - 1) / 2 and x zero outside the image,
 *          the oracle's blur operator
 *  psf     HOST, K x K FP32, row-major
 *  reps    >= 1; each image stays in shared memory between applications
 * Limits: K = 9; nx a positive multiple of 16; the image must fit shared
 * memory (64 x 64 fits both engines).  Returns MIRAGE_ERR_ARG or
 * MIRAGE_ERR_UNSUPPORTED otherwise (text in mirage_blur_last_error).  If a
 * tensor-core completion wait runs out (about a second), the affected
 * images are written as NaN.  Asynchronous on `stream`. */
#define MIRAGE_BLUR_FFMA 0
#define MIRAGE_BLUR_TC_TF32 1
int mirage_psf_blur(int engine, const float* img, float* out, int n, int nx, int ny, const float* psf, int K,
                    int reps, void* stream);
const char* mirage_blur_last_error(void);

/* FP32 FMA-pipe microbenchmark on `device`: sixteen independent FMA chains
 * per thread on every SM, timed with CUDA events after a warm-up launch.
 * Writes the sustained FP32 TFLOP/s and the flops per clock per SM at the
 * device's maximum SM clock (nominal 256 = 128 lanes x 2).  The binding
 * roof of the CGLS kernels, measured rather than derived.  Synchronous;
 * allocates and frees a small output buffer. */
int mirage_measure_ffma(int device, double* tflops, double* flop_per_clk_sm);

#ifdef __cplusplus
}
#endif
#endif /* MIRAGE_H */
