/*
 * qmcslice.h - C ABI of the GB300 (sm_103a) QMC-slicing fast kernel summation.
 *
 * Method: Hertrich, Jahn, Quellmalz, "Fast Summation of Radial Kernels via QMC
 * Slicing", arXiv 2410.01316.  The library computes the kernel sums
 *
 *     s_m = sum_n w_n F(|x_n - y_m|),   m = 1..M                (Sec. 1, eq. kernel_sum)
 *
 * by slicing (Sec. 2.1, eq. kernel_sum_sliced): average over P directions
 * xi_p of one-dimensional sums of the projections <x_n, xi_p>, <y_m, xi_p>
 * with the sliced basis function f, each evaluated by one-dimensional fast
 * Fourier summation (App. C, eq. 1d_sum_fourier; App. G, eq. Fourier-slicing):
 *
 *     a_{n,p} = tau <x_n, xi_p>,   b_{m,p} = tau <y_m, xi_p>
 *     s_m ~= (1/P) sum_p Re sum_{k=-N_ft/2}^{N_ft/2-1} c_k e^{2 pi i k b_{m,p}}
 *                            sum_n w_n e^{-2 pi i k a_{n,p}}
 *
 * The inner sums are computed with an oversampled grid of G = 2 N_ft cells
 * per slice (window spreading, FFT, multiplication by c_k over the squared
 * window transform, inverse FFT, window interpolation).
 *
 * Conventions shared by every entry point:
 *  - Point arrays are row-major FP32: x is N x d, y is M x d; w has N entries,
 *    s has M entries.  Pointers passed to qs_sum / qs_grad are DEVICE pointers
 *    owned by the caller; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Argument errors are returned immediately.  Data errors detected on the
 *    device (a projection outside the half period, a NaN/Inf input, an
 *    exhausted wait) are recorded in the plan's device error flag and
 *    returned by qs_check.
 *  - No entry point throws, aborts or prints.  qs_last_error() returns a
 *    human-readable message for the most recent failure on this thread.
 *  - A plan may be used from one host thread at a time; calls on the same
 *    plan must be ordered on one stream (they share the plan's workspace).
 */
#ifndef QMCSLICE_H
#define QMCSLICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_plan_s* qs_plan;

typedef enum {
    QS_OK = 0,
    QS_ERR_ARG = 1,         /* invalid argument (NULL pointer, bad size, bad enum) */
    QS_ERR_RANGE = 2,       /* a projection |tau <x, xi>| exceeded 1/2: radius too small */
    QS_ERR_NONFINITE = 3,   /* NaN or Inf in x, y or w */
    QS_ERR_OOM = 4,         /* device or host allocation failed (plan creation only) */
    QS_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    QS_ERR_UNSUPPORTED = 6, /* valid but not supported configuration */
    QS_ERR_TIMEOUT = 7      /* a bounded device wait gave up */
} qs_status;

/* Radial kernels F (Table tab:kernels). */
typedef enum {
    QS_GAUSS = 0,   /* F(r) = exp(-r^2 / (2 sigma^2)),  kparam = sigma */
    QS_LAPLACE = 1, /* F(r) = exp(-alpha r),            kparam = alpha */
    QS_NEGDIST = 2, /* F(r) = -r (Riesz r = 1),          kparam unused  */
    QS_MATERN = 3,  /* F(r) = 2^{1-nu}/Gamma(nu) (sqrt(2 nu) r/beta)^nu K_nu(sqrt(2 nu) r/beta),
                       kparam = beta > 0, kparam2 = nu > 0 */
    QS_RIESZ = 4,   /* F(r) = -r^q (generalised Riesz), kparam = q in (0, 2) */
    QS_TPS = 5      /* F(r) = r^2 log r (thin plate spline), kparam unused */
} qs_kernel;

/* Direction designs (Sec. 4.1, "QMC Sequences"). */
typedef enum {
    QS_DIR_USER = 0,       /* caller supplies P x d unit rows in dirs_host */
    QS_DIR_FIBONACCI = 1,  /* spherical Fibonacci points, d = 3 only */
    QS_DIR_ORTHOGONAL = 2, /* first P columns of ceil(P/d) Haar-orthogonal matrices */
    QS_DIR_IID = 3,        /* iid uniform on the sphere */
    QS_DIR_DISTANCE = 4,   /* distance QMC design: QS_DIR_ORTHOGONAL (seeded) refined by
                              qs_distance_design (300 steps, lr 0.05/sqrt(d)) at plan creation;
                              plans only (qs_directions refuses it: it needs the GPU) */
    QS_DIR_SOBOL = 5       /* Sobol' points (qs_sobol_points, digitally shifted by `seed`; seed 0 =
                              unshifted) mapped through the inverse normal CDF per coordinate and
                              normalised; d <= 4096 */
} qs_dirs;

/* Precision / form of the projection step a = tau X Xi^T. */
typedef enum {
    QS_PROJ_AUTO = 0,       /* fused for d <= 4, FP32 for d < 64, BF16x3 from d = 64 */
    QS_PROJ_FP32 = 1,       /* FP32 SIMT GEMM into a P x N workspace */
    QS_PROJ_FP32_FUSED = 2, /* FP32 dot products inside spread / interpolation (d <= 64) */
    QS_PROJ_BF16X3 = 3,     /* tensor-core GEMM, x = hi + lo split in BF16, three products */
    QS_PROJ_TF32 = 4        /* tensor-core GEMM in TF32 */
} qs_proj;

/* Window of the oversampled grid (App. C; the paper uses NFFT's default and does not name it). */
typedef enum {
    QS_WINDOW_ES = 0,      /* exponential of semicircle exp(beta (sqrt(1 - (v/m)^2) - 1)), beta = 2.3 W */
    QS_WINDOW_KB = 1       /* Kaiser-Bessel, sinh form: sinh(b sqrt(m^2 - v^2)) / sqrt(m^2 - v^2), b = 3 pi / 2 */
} qs_window_kind;

typedef struct {
    int d;                 /* dimension, >= 1 */
    qs_kernel kernel;
    double kparam;         /* sigma (Gauss), alpha (Laplace), beta (Matern), q (Riesz); else ignored */
    int P;                 /* number of slices, >= 1 */
    qs_dirs dirs;
    uint64_t seed;         /* seed for QS_DIR_ORTHOGONAL / QS_DIR_IID */
    const float* dirs_host;/* P x d host array for QS_DIR_USER (copied), else NULL */
    int n_ft;              /* number of Fourier coefficients, power of two, 16 .. 8192 */
    int window;            /* window taps W per point: 6, 8, 10 or 12 (0 = 8) */
    double oversampling;   /* grid oversampling sigma_os; only 2.0 is supported (0 = 2) */
    double radius;         /* R >= max|x_n| + max|y_m| (App. G, eq. radius_xy), > 0 */
    qs_proj proj;
    int64_t max_n, max_m;  /* largest N and M the plan will be called with */
    double kparam2;        /* nu (Matern); else ignored */
    int window_kind;       /* qs_window_kind (0 = QS_WINDOW_ES); W = 2m taps either way */
} qs_plan_desc;

/*
 * Create a plan: the rescaling factor tau (App. C Step 1 for Gauss / Laplace /
 * Matern: tau = min(T/R, 1/(2 g_max)) with T = 0.3 / 0.1 / 0.2; App. G for the
 * negative distance, generalised Riesz and thin plate spline kernels: tau =
 * 1/(2R)), the directions, the Fourier coefficients c_k in FP64 (App. C Step 2:
 * closed-form transforms on the device for Gauss / Laplace / Matern / negative
 * distance; for Riesz and the thin plate spline, which have no classical
 * transform, the integrals of the periodised 1D function over one period by
 * host quadrature), the window tables (tap polynomials of the chosen window
 * and its Fourier transform by quadrature of those polynomials), and all
 * device workspace.  Runs on the
 * current CUDA device and synchronises it.  On success *out holds the plan.
 * Errors: QS_ERR_ARG, QS_ERR_UNSUPPORTED, QS_ERR_OOM, QS_ERR_CUDA.
 */
qs_status qs_plan_create(qs_plan* out, const qs_plan_desc* desc);

/* Release the plan and its device memory.  Synchronises the device.  NULL is a no-op. */
qs_status qs_plan_destroy(qs_plan plan);

/*
 * Query the plan: tau (double), the grid size G, the number of slices and the
 * device pointer of the FP32 P x d direction array used by the sums.  Any
 * output pointer may be NULL.  The direction pointer stays valid until
 * qs_plan_destroy.
 */
qs_status qs_plan_info(qs_plan plan, double* tau, int* grid_size, int* P, const float** dirs_dev);

/*
 * Copy the plan's FP32 directions (P x d, row-major) into a host buffer.
 * Synchronous.
 */
qs_status qs_plan_directions(qs_plan plan, float* dirs_host);

/*
 * s = fast sliced kernel sum (the pipeline described at the top of this file).
 * x: N x d, w: N (NULL = all weights one), y: M x d, s: M; all device memory.
 * N <= max_n, M <= max_m.  Asynchronous on `stream`; allocates nothing and
 * does not synchronise.  N = 0 gives s = 0; M = 0 is a no-op.
 * Errors returned: QS_ERR_ARG, QS_ERR_CUDA (launch failure).  Data errors:
 * qs_check.
 */
qs_status qs_sum(qs_plan plan, const float* x, int64_t N, const float* w,
                 const float* y, int64_t M, float* s, void* stream);

/*
 * Gradients of L = sum_m v_m s_m with s = qs_sum(x, w, y) (the derivative of
 * the sliced Fourier sum of Sec. 2.1 / App. C; its use for MMD gradient flows
 * is App. H).  With g(t) = Re sum_k c_k e^{2 pi i k t} (even) and g' odd:
 *   gy[m] = dL/dy_m = (tau/P) v_m sum_p xi_p sum_n w_n g'(b_{m,p} - a_{n,p})
 *   gx[n] = dL/dx_n = (tau/P) w_n sum_p xi_p sum_m v_m g'(a_{n,p} - b_{m,p})
 *   gw[n] = dL/dw_n = (1/P) sum_p sum_m v_m g(a_{n,p} - b_{m,p})
 * computed by the same spread / FFT / interpolation pipeline with the filter
 * 2 pi i k c_k / psi^2 and a back-projection onto the directions (x and w
 * swap roles with y and v).  The unfused projection forms (QS_PROJ_FP32,
 * QS_PROJ_BF16X3, QS_PROJ_TF32) write the derivative values of every
 * (point, slice) pair over the plan's projection buffer and back-project them
 * by a GEMM (points x P)(P x d) with compensated slice-chunk sums; the fused
 * form, which has no projection buffer, sums the back-projection inside the
 * interpolation per component and so needs d <= 32.  x: N x d,
 * w: N (NULL = ones), y: M x d, v: M (NULL = ones), gx: N x d, gw: N,
 * gy: M x d; all device memory; any output may be NULL to skip it.
 * Asynchronous on `stream`, allocates nothing.  Errors: QS_ERR_ARG,
 * QS_ERR_UNSUPPORTED (fused form with d > 32), QS_ERR_CUDA; data errors via
 * qs_check.
 */
qs_status qs_grad(qs_plan plan, const float* x, int64_t N, const float* w, const float* y, int64_t M,
                  const float* v, float* gx, float* gw, float* gy, void* stream);

/*
 * The projection step alone (Sec. 2.1, eq. kernel_sum_sliced; App. C Step 1):
 * u_out[p * ldu + n] = G tau <x_n, xi_p> for p < P, n < N, computed in the
 * plan's projection form (FP32, BF16x3 or TF32; the fused form uses FP32).
 * x: N x d device memory; u_out: P x ldu device memory, ldu >= N.
 * Asynchronous on `stream`; uses the plan's workspace, allocates nothing.
 */
qs_status qs_project(qs_plan plan, const float* x, int64_t N, float* u_out, int64_t ldu, void* stream);

/*
 * Same sum from HOST buffers: copies x, w, y into plan-owned device staging
 * buffers, computes the sum, copies s back into the host buffer and
 * synchronises `stream`.  The copies in run on a plan-owned copy stream in
 * row chunks (at most 8 for x and 2 for y, after the work already queued on
 * `stream`), and each chunk is projected on `stream` as soon as it has
 * landed (each target chunk also interpolated), so the transfers overlap the
 * projections, the spread and the interpolation; the result is the one
 * qs_sum computes, bit for bit.  With
 * stage timing on (qs_set_timing) or N == 0 the copies run first, on
 * `stream`.  Pinned host memory gives the fastest copies; the host buffers
 * must stay unchanged until the call returns.  Returns the data-error status
 * as qs_check would.
 */
qs_status qs_sum_host(qs_plan plan, const float* x_host, int64_t N, const float* w_host,
                      const float* y_host, int64_t M, float* s_host, void* stream);

/*
 * Synchronise `stream`, read and clear the plan's device error flag.
 * Returns QS_OK, QS_ERR_RANGE, QS_ERR_NONFINITE, QS_ERR_TIMEOUT or QS_ERR_CUDA.
 */
qs_status qs_check(qs_plan plan, void* stream);

/* Static English description of a status code. */
const char* qs_status_string(qs_status status);

/* Message describing the most recent failure on the calling thread ("" if none). */
const char* qs_last_error(void);

/*
 * Host-only direction generator (no GPU needed): writes P x d unit rows into
 * out_host for QS_DIR_FIBONACCI (d = 3), QS_DIR_ORTHOGONAL, QS_DIR_IID or
 * QS_DIR_SOBOL (Sec. 4.1).  Deterministic in `seed`.
 */
qs_status qs_directions(qs_dirs kind, int d, int P, uint64_t seed, float* out_host);

/*
 * The Sobol' sequence behind QS_DIR_SOBOL (Sec. 4.1, "QMC Sequences"): writes
 * points i = 0 .. P-1 of a d-dimensional Sobol' sequence, u[i * d + j] =
 * (x_ij + 1/2) / 2^32 in (0, 1), into the host array out_host (P x d doubles,
 * caller-owned).  Coordinate 0 is the van der Corput sequence; coordinate
 * j >= 1 uses the j-th primitive polynomial over GF(2) (ordered by degree,
 * then coefficients) with 32-bit direction numbers; points in Gray-code
 * (Antonov-Saleev) order.  The first 2^m points of
 * every coordinate hold one point in each interval [k 2^-m, (k+1) 2^-m), and
 * coordinates 0 and 1 form a (0, m, 2)-net.  seed != 0 applies a seeded
 * random digital shift (XOR per coordinate), which keeps these properties.
 * Errors: QS_ERR_ARG (NULL output, P < 1, d outside 1 .. 4096).
 */
qs_status qs_sobol_points(int d, int P, uint64_t seed, double* out_host);

/*
 * Stage timing for benchmarks.  While enabled, qs_sum records a CUDA event on
 * its stream between consecutive stages.  qs_stage_times waits for the events
 * of the most recent qs_sum call on this plan and writes up to n (<= 7) stage
 * durations in milliseconds:
 *   [0] operand split of x (tensor-core forms)   [1] projection GEMM of x
 *   [2] weight bound + spread + FFT filter        [3] operand split of y
 *   [4] projection GEMM of y                       [5] interpolation
 *   [6] slice reduction
 * Stages the plan's form does not run report 0.  In the tensor-core forms
 * with d >= 256 stage [3] runs on a plan-owned side stream concurrently with stage [1]
 * (qs_sum forks it after stage [0] and joins it before stage [4]) and
 * reports its own duration, which is off the critical path.
 * Enabling creates the events (host-side driver objects, no device memory).
 * Do not enable while a stream that the plan uses is being captured into a
 * CUDA graph.
 */
qs_status qs_set_timing(qs_plan plan, int enable);
qs_status qs_stage_times(qs_plan plan, float* ms, int n);

/*
 * The sum for callers that cannot allocate device memory.  (The paper has
 * no counterpart; this is a deployment entry point.)
 *
 * Some callers cannot call cudaMalloc: code running under a framework whose
 * caching allocator owns the device memory, loops that must not stall on an
 * allocation, or plugins that are handed their buffers and nothing else.
 * Plan creation allocates, so they cannot hold a plan.  qs_sum_noalloc takes
 * the plan description directly and keeps every intermediate in one static
 * device array of 16 MiB that the library reserves on each GPU it is loaded
 * on, until the process exits.  It allocates nothing.
 *
 * desc: as for qs_plan_create; dirs, seed, dirs_host, max_n and max_m are
 *       ignored and proj must be QS_PROJ_AUTO or QS_PROJ_FP32_FUSED (FP32 dot
 *       products inside the spread and interpolation; d <= 64).  QS_RIESZ and
 *       QS_TPS, whose coefficients need host quadrature, return
 *       QS_ERR_UNSUPPORTED.
 * dirs_dev: P x d FP32 directions in device memory (caller-owned); a
 *       non-finite entry makes the call return QS_ERR_NONFINITE.
 * x, w, y, s: as for qs_sum (device memory, w may be NULL).
 * Sizes: P * 2 n_ft grid values, the tables and the slice partial sums must
 * fit in the 16 MiB array (e.g. P = 1024 slices with n_ft = 1024 and M up to
 * about a million targets); larger problems return QS_ERR_UNSUPPORTED with a
 * message giving the bytes needed.  N and M are otherwise unbounded.
 * Result: where the slice partial sums fit at the slice-group count qs_sum
 * uses, the result is bit for bit that of qs_sum on a QS_PROJ_FP32_FUSED plan
 * with the same description and directions (same tables, same kernels).
 * Synchronous: waits for `stream` and returns the data-error status that
 * qs_check would return.  The window tables are computed on the host once
 * per (window, grid size) and kept in a small static cache.
 * The first call on a device does a one-time set-up: it looks up the
 * array's device address (and looks it up again after the device's context
 * has been reset); make that first call before any stream capture begins.
 * All calls share the array and it keeps the last call's contents: calls
 * whose GPU work overlaps (other streams or threads on the same device) race
 * and must be serialised by the caller.
 */
qs_status qs_sum_noalloc(const qs_plan_desc* desc, const float* dirs_dev, const float* x, int64_t N,
                         const float* w, const float* y, int64_t M, float* s, void* stream);

/*
 * Batched sums.  Many independent problems, each with its own plan (its own
 * d <= 64, P, N_ft, kernel and directions; all plans must share the window
 * width), run in ONE persistent launch that drains a queue of
 * (problem, slice) spread items followed by (problem, target block)
 * interpolation items, largest problems first.  Projections are FP32: SIMT
 * GEMM tile items before the spread items for d > 4, dot products inside the
 * items for d <= 4.  Each target's slice sum is formed in slice order by one
 * thread, so results do not depend on the tiling.
 *
 * qs_batch_create: plans are borrowed (they must outlive the batch); their
 *   workspaces hold the intermediate grids.  Allocates the batch's
 *   descriptor table (pinned host + device).
 * qs_sum_batched: probs[k] is the problem of plans[k] (device pointers as for
 *   qs_sum; w may be NULL).  Asynchronous on `stream`.  The problem table is
 *   uploaded from the batch's pinned staging; outside graph capture the call
 *   first waits until the previous call's upload has executed.  A captured
 *   call replays with the table of the call that was captured.
 * qs_batch_check: synchronises `stream` and returns the worst data-error
 *   status of the batch's plans (clearing their flags).
 * qs_batch_set_tiling: largest number of targets per thread of the
 *   interpolation items (1, 2 or 4; the default 4 is capped by d so that a
 *   block's coordinates fit a 64 KB shared tile).
 */
typedef struct qs_batch_s* qs_batch;
typedef struct {
    const float* x;  /* N x d sources */
    int64_t N;
    const float* w;  /* N weights or NULL */
    const float* y;  /* M x d targets */
    int64_t M;
    float* s;        /* M outputs */
} qs_problem;
qs_status qs_batch_create(qs_batch* out, const qs_plan* plans, int nprob);
qs_status qs_batch_destroy(qs_batch batch);
qs_status qs_sum_batched(qs_batch batch, const qs_problem* probs, void* stream);
qs_status qs_batch_check(qs_batch batch, void* stream);
qs_status qs_batch_set_tiling(qs_batch batch, int targets_per_thread);
/*
 * Execution mode of qs_sum_batched.  QS_BATCH_PERSISTENT (the default): the
 * one persistent launch described above.  QS_BATCH_CONCURRENT: every problem
 * runs its own plan's qs_sum pipeline (the plan's projection form, spread
 * family and interpolation) on one of 8 streams owned by the batch, problems
 * assigned largest first to the least-loaded stream; the streams are forked
 * from and joined to `stream`, so the call is ordered on `stream` and can be
 * captured into a CUDA graph.  Each problem's result is then bit for bit
 * that of qs_sum on its plan.  QS_ERR_ARG for other values.
 */
typedef enum { QS_BATCH_PERSISTENT = 0, QS_BATCH_CONCURRENT = 1 } qs_batch_mode;
qs_status qs_batch_set_mode(qs_batch batch, int mode);
/*
 * Time qs_sum_batched on these problems in the persistent mode with 1, 2 and
 * 4 targets per thread of the interpolation items and in the concurrent mode
 * (best of two after a warm-up, CUDA events on `stream`), keep the fastest in
 * the batch and write it to *chosen (may be NULL): 1, 2 or 4 for the
 * persistent kernel with that tiling, 0 for the concurrent mode.  The tilings
 * give bitwise identical results; the modes differ within the sums'
 * accuracy.  Synchronous; the problems' outputs are written (several times).
 */
qs_status qs_batch_autotune(qs_batch batch, const qs_problem* probs, int* chosen, void* stream);

/*
 * Tuning.  The spread stage has variants in two families, fixed by the grid
 * size G and the window W: the moment family (4: one bin table; 5: a 32-bin
 * lane-interleaved window plus the table) where its shared memory fits two
 * CTAs per SM (G <= 2048 for W <= 8, G <= 1024 for W >= 10), the tap family
 * otherwise (0..2: one point per thread with 1, 2 or 4 lane-private grid
 * copies; 3: a 32-cell window with one column per thread plus one grid).
 * Within a family the variants produce bitwise identical results and differ
 * only in speed, which depends on how the projections cluster.
 * qs_plan_autotune runs the spread of the given sources once per variant of
 * the family (timed with CUDA events on `stream`, best of 3 after a warm-up),
 * keeps the fastest in the plan and writes its index to *chosen (may be
 * NULL).  Synchronous.  qs_plan_set_variant fixes a variant directly
 * (QS_ERR_ARG if out of range or of the other family).
 */
qs_status qs_plan_autotune(qs_plan plan, const float* x, int64_t N, const float* w, int* chosen, void* stream);
/*
 * Projection GEMM form by timing (tensor-core plans): runs the projection of
 * the N points in x (device, N x d) with one CTA per SM and, where two-CTA
 * clusters can be resident, on SM pairs (best of 3 after a warm-up, CUDA
 * events on `stream`) and keeps the faster (*chosen = pair, may be NULL).
 * Unlike the spread variants, the two forms may differ in the last bits of
 * the projections (the tensor cores' internal accumulation order; both stay
 * within the rounding bound of the form).  Synchronous.  QS_ERR_UNSUPPORTED
 * for plans without a tensor-core projection.
 *
 * Autotune cache: qs_plan_autotune and qs_plan_autotune_gemm record their
 * choice under the plan's shape class (d rounded up to a power of two, N_ft,
 * P rounded up to a power of two, projection form, window width); plans
 * created later in the process for the same class start with the recorded
 * choices.  The cache can be written to and read from a text file, cleared,
 * and queried for its number of entries.
 */
qs_status qs_plan_autotune_gemm(qs_plan plan, const float* x, int64_t N, int* chosen, void* stream);
qs_status qs_tune_cache_save(const char* path);
qs_status qs_tune_cache_load(const char* path);
qs_status qs_tune_cache_clear(void);
int qs_tune_cache_size(void);
qs_status qs_plan_set_variant(qs_plan plan, int spread_variant);
/* Variants of the plan's family (bit v of *available set for variant v) and
 * the variant in use (*current); either pointer may be NULL.  Host only. */
qs_status qs_plan_variants(qs_plan plan, unsigned int* available, int* current);

/*
 * Projection GEMM form of a tensor-core plan (QS_PROJ_BF16X3 / QS_PROJ_TF32),
 * i.e. how the projections <x_n, xi_p> of Sec. 2.1 eq. kernel_sum_sliced are computed:
 * pair = 0 runs one CTA per SM on 128-point x 256-slice tiles; pair = 1 runs
 * clusters of two CTAs on SM pairs (tcgen05 cta_group::2) on 256-point x
 * 256-slice tiles, which halves the shared-memory reads of the directions per
 * SM.  qs_plan_create picks pair = 1 for d >= 256 (where the GEMM is bound by
 * the tensor pipe rather than by its stores of U) wherever such clusters can
 * be resident.  Both give the same projections up to the order of the tensor cores'
 * internal FP32 sums.  QS_ERR_UNSUPPORTED for pair = 1 on other projection
 * forms or where two-CTA clusters of the kernel cannot be resident;
 * QS_ERR_ARG for other values.  qs_plan_gemm reports the form in use (0 / 1)
 * in *pair and, if ctas is not NULL, the CTAs a full-size launch of it runs
 * (SM count, or twice the resident two-CTA clusters).  Host only; affects
 * later calls.
 */
qs_status qs_plan_set_gemm(qs_plan plan, int pair);
qs_status qs_plan_gemm(qs_plan plan, int* pair, int* ctas);

/*
 * Sorting slicing for the negative distance kernel (Sec. 2.1, eq.
 * kernel_sum_sliced with f(t) = -c_d |t|; the sorting evaluation the paper
 * uses for this kernel): the sliced sum over the plan's directions computed
 * exactly, without the Fourier truncation, by sorting each slice's source
 * and target projections (FP32, from the FP32 SIMT projection) together and
 * scanning prefix sums of w and w a in 64-bit fixed point (exact integer
 * sums with per-slice scales, combined per target in error-free FP32
 * arithmetic): sum_n w_n |b - a_n| = b (2 W_< - W) - (2 S_< - S).
 * Arguments as for qs_sum.  Needs a QS_NEGDIST plan with d <= 64
 * (QS_ERR_UNSUPPORTED otherwise).  The first call allocates the plan's
 * sorting workspace (about 21 CS (max_n + max_m) + 4 CS max_m + 512 max_m
 * bytes, CS = min(P, 128) slices per chunk) and so synchronises; later
 * calls are asynchronous and allocate nothing.  Data errors (non-finite
 * projections or weights) go to the device flag.
 */
qs_status qs_sum_sorted(qs_plan plan, const float* x, int64_t N, const float* w, const float* y, int64_t M,
                        float* s, void* stream);
/*
 * Gradient in the targets of L = sum_m v_m s_m for the same exact sliced sum:
 *   gy[m] = v_m (-c_d / P) sum_p (sum_n w_n sign(<xi_p, y_m - x_n>)) xi_p
 * (M x d, row-major, device; v may be NULL for all ones), from the same sort
 * (2 W_< - W per target and slice) and a fixed-order compensated sum over the
 * slices.  A source whose projection equals a target's exactly counts as
 * below it (one-sided subgradient).  Requirements, workspace and errors as
 * for qs_sum_sorted.
 */
qs_status qs_grad_sorted(qs_plan plan, const float* x, int64_t N, const float* w, const float* y, int64_t M,
                         const float* v, float* gy, void* stream);

/*
 * Distance QMC designs (Sec. 2.3, eq. distance-mmd with s = d/2; Sec. 4.1,
 * "Distance"; the symmetric energy of eq. distance-sym):
 *   E_sym(xi) = -2 sum_{p,q} (|xi_p - xi_q| + |xi_p + xi_q|)
 * over P unit directions in R^d, minimised by Adam (beta1 0.9, beta2 0.999)
 * on the gradient's component tangent to the sphere, the step annealed from
 * lr to lr/100 (cosine) over the `iters` steps, every step followed by
 * renormalising the rows.
 *
 * qs_distance_design: runs `iters` steps on the P x d FP32 rows in dirs_dev
 * (device, caller-owned, updated in place; start from any unit rows, e.g.
 * QS_DIR_ORTHOGONAL); if energy is not NULL it receives E_sym of the result.
 * qs_distance_energy: E_sym of the rows in dirs_dev and, if grad_dev is not
 * NULL, its Euclidean gradient dE/dxi (P x d device array, caller-owned).
 * Both contractions of a step (the Gram matrix and (B - A) Xi, P x P x d
 * each) run on the tcgen05 GEMM in BF16x3 (split operands, FP32
 * accumulation), the second as up to 20 inner ranges on streams of the
 * routine's own; the weights of near-parallel or near-antipodal pairs
 * (|c_pq| > 1/2) take |xi_p -+ xi_q|^2 from the rows instead of 2 -+ 2 c_pq.
 * d up to ~58000.  Both are set-up routines, not part of the sum: they
 * allocate and free a workspace of about 8 P^2 + (20 + 4 ks) P d' bytes
 * (d' = d rounded up to 128, ks <= 20 the ranges) on the current device,
 * run on `stream` and return when it is done.  Errors: QS_ERR_ARG (NULL pointer,
 * d or P < 1, iters < 0, lr <= 0), QS_ERR_UNSUPPORTED (P^2 beyond 2^31),
 * QS_ERR_OOM, QS_ERR_CUDA (also when a GEMM wait ran out; the device flag of
 * plans is not involved).
 */
qs_status qs_distance_design(float* dirs_dev, int d, int P, int iters, double lr, double* energy, void* stream);
qs_status qs_distance_energy(const float* dirs_dev, int d, int P, double* energy, float* grad_dev, void* stream);

/* Library version string. */
const char* qs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QMCSLICE_H */
