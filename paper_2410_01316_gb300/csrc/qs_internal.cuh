// Internal declarations shared by the CUDA sources of the qmcslice library.
//
// Notation (arXiv 2410.01316, App. C and App. G): a plan holds P directions
// xi_p, the rescaling factor tau, N_ft Fourier coefficients c_k and an
// oversampled grid of G = 2 N_ft cells per slice.  Projections are kept in
// grid units, u = G tau <x, xi_p>, so one grid cell has width 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qmcslice.h"

// stages timed by qs_set_timing / qs_stage_times
#define QS_NUM_STAGES 7
#define QS_HOST_CHUNKS 8    // most row chunks of x in the qs_sum_host pipeline
#define QS_HOST_Y_CHUNKS 2  // row chunks of y (measured: 2.33 ms end to end for 2, 2.38 for 3, 2.76 for 8)

// device error flag bits (qs_check maps them to qs_status)
#define QS_FLAG_RANGE 1u
#define QS_FLAG_NONFINITE 2u
#define QS_FLAG_TIMEOUT 4u

// Window: exponential of semicircle psi(v) = exp(beta (sqrt(1 - (v/m)^2) - 1))
// on |v| < m = W/2 grid cells.  Each point touches W cells; the W tap values
// are piecewise polynomials of the fractional offset.
constexpr int QS_MAX_W = 12;
constexpr int QS_MAX_HALF = QS_MAX_W / 2;
constexpr int QS_MAX_TERMS = QS_MAX_HALF + 1;  // terms per even / odd part
constexpr int QS_MAX_G = 16384;                // grid cells per slice (64 KB shared)
constexpr int QS_FUSED_MAX_D = 64;             // largest d of the fused form
constexpr int QS_GRAD_MAX_D = 32;              // largest d of the fused form's gradients (per-component sums)
constexpr int QS_BATCH_MAX_D = 64;             // largest d of a batched problem
constexpr int QS_SOBOL_MAX_D = 4096;           // largest d of the Sobol' directions
constexpr int QS_BATCH_STREAMS = 8;            // streams of a batch's concurrent mode

// Spread kernel variants, in two families fixed by (G, W): the moment family
// where its table fits two CTAs per SM, the tap family otherwise.  Within a
// family the variants give bitwise identical grids and are chosen by timing.
enum {
    QS_SPREAD_POINT1 = 0,       // taps: point per thread, one grid
    QS_SPREAD_POINT2 = 1,       // taps: two lane-private grid copies
    QS_SPREAD_POINT4 = 2,       // taps: four copies
    QS_SPREAD_THREAD32 = 3,     // taps: thread-private 32-cell window columns + one grid
    QS_SPREAD_MOMENT = 4,       // moments: one bin table
    QS_SPREAD_MOMENTWIN32 = 5,  // moments: lane-interleaved 32-bin window + the bin table
    QS_SPREAD_NVARIANTS = 6
};

// Degree of the tap polynomials: W - 1 from W = 8 on (the tap error is then
// ~4e-8, limited by the square-root edge of the window anyway), W + 1 below.
__host__ __device__ constexpr int qs_tap_degree(int W) { return W >= 8 ? W - 1 : W + 1; }
// Terms of each even / odd part (the degree is odd).
__host__ __device__ constexpr int qs_tap_terms(int W) { return (qs_tap_degree(W) + 1) / 2; }

constexpr int QS_SPREAD_PAD = 16;    // overflow cells of the linear spread grid
constexpr int QS_MOMENT_WIN = 32;    // bins of the lane-interleaved moment window

// Moments per point of the moment spread: the tap polynomials' degree + 1.
__host__ __device__ constexpr int qs_moment_count(int W) { return qs_tap_degree(W) + 1; }

// Shared bytes of the moment spread: the bin table ((G + 16) rows of K + 1
// ints) and the larger of the lane window and the float grid it becomes.
inline size_t qs_moment_smem(int G, int W, bool window)
{
    const size_t K = (size_t)qs_moment_count(W), cs = (size_t)G + QS_SPREAD_PAD;
    const size_t lw = window ? (size_t)QS_MOMENT_WIN * K * 32 * 4 : 0, grid = cs * 4;
    return cs * (K + 1) * 4 + (lw > grid ? lw : grid);
}
// The moment family is used when both its variants fit two CTAs per SM.
inline bool qs_spread_moments(int G, int W) { return qs_moment_smem(G, W, true) <= (size_t)113 * 1024; }
inline int qs_spread_default(int G, int W) { return qs_spread_moments(G, W) ? QS_SPREAD_MOMENT : QS_SPREAD_POINT1; }
inline bool qs_spread_variant_ok(int G, int W, int v)
{
    return v >= 0 && v < QS_SPREAD_NVARIANTS && (v >= QS_SPREAD_MOMENT) == qs_spread_moments(G, W);
}

// Tap polynomials.  For tap j of the first half (0 <= j < m), with the
// centred fractional offset s in [-1/2, 1/2]:
//   psi(s + m - 1/2 - j)         = E_j(s^2) + s O_j(s^2)
//   psi(s + m - 1/2 - (W-1-j))   = E_j(s^2) - s O_j(s^2)   (psi is even)
struct qs_window {
    float e[QS_MAX_HALF][QS_MAX_TERMS];
    float o[QS_MAX_HALF][QS_MAX_TERMS];
};

// Everything a launch of the sum pipeline needs (passed by value).
struct qs_launch {
    int d, P, G, n_ft;
    int64_t N, M;
    int64_t m_base, m_end;  // targets [m_base, m_end) of an interpolation launch (0, M by default)
    int64_t ldU;          // row stride (elements) of the P x ldU projection workspace
    float half_G;         // |u| must stay <= G/2 (the half period)
    const float* xi_s;    // P x d, directions scaled by G tau
    const float* D;       // G/2 + 1 filter weights c_k / psi^(k/G)^2, 0 beyond N_ft/2
    const float2* tw;     // G/2 twiddles e^{-2 pi i t / G}
    float* H;             // P x G filtered grids
    float* U;             // P x ldU projections (unfused forms)
    float* part;          // 2 x S x M partial slice sums (hi, lo)
    int S;                // number of slice groups of the interpolation
    unsigned int* flag;   // device error flag
    float* wscale;        // [0] = 2^30 / sum|w| (fixed-point scale of the grids), [1] = its inverse
    int spread_variant;   // QS_SPREAD_* (all variants give bitwise identical grids)
    qs_window win;
    // tap polynomials in monomials of t = 2 s: tap_j(t) = sum_k atab[j K + k] t^k, K = qs_moment_count(W)
    // (qs_fill_atab); in the launch parameters, so the interpolation's bin expansion takes them as
    // constant operands
    float atab[QS_MAX_W * QS_MAX_W];
};

struct qs_plan_s {
    int device;
    int sm_count;
    qs_plan_desc desc;    // copy; dirs_host cleared
    qs_proj proj;         // resolved form
    double tau;
    int G, W;
    int window_kind;      // QS_WINDOW_ES / QS_WINDOW_KB
    int64_t ldU;
    int S_max;            // slice-group capacity of the partial buffer
    size_t U_elems;
    qs_window win;
    int spread_variant;   // fixed by qs_set_spread_variant or the first timed tuning
    // device buffers
    float* d_dirs;        // P x d
    float* d_dirs_s;      // P x d scaled by G tau
    double* d_c;          // n_ft coefficients c_k, k = -n_ft/2 .. n_ft/2-1
    double* d_psihat;     // n_ft/2 + 1 window transform values (FP64)
    float* d_D;           // G/2 + 1
    float2* d_tw;         // G/2
    float* d_U;
    float* d_H;
    float* d_part;
    unsigned int* d_flag;
    float* d_wscale;      // 2 floats, written by the weight-bound kernel of each sum
    // gradients: derivative filter, second grid; per-component partials (fused form, d <= 32)
    float* d_Dd;          // G/2 + 1
    float* d_H2;          // P x G
    float* d_gpart;       // 2 x (S M)max x d
    size_t gpart_elems;
    // staging for qs_sum_host
    float* d_x;
    float* d_w;
    float* d_y;
    float* d_s;
    // tensor-core projection operands: BF16 hi/lo split (BF16x3) or TF32
    // rounding of the scaled directions and of the points being projected
    int ldk;              // row stride (elements) of the operand copies
    void* d_xi_hi;        // P x ldk
    void* d_xi_lo;        // P x ldk (BF16x3 only)
    void* d_xs_hi;        // max(max_n, max_m) x ldk staging of the points (the sources, qs_project, host chunks)
    void* d_xs_lo;        // (BF16x3 only)
    void* d_ys_hi;        // max_m x ldk staging of the targets (split while the sources' GEMM runs)
    void* d_ys_lo;        // (BF16x3 only)
    void* d_sortws = nullptr;  // sorting-slicing workspace, allocated by the first qs_sum_sorted
    // CUtensorMap: points hi/lo (128-row boxes), directions hi/lo (256-row boxes),
    // directions hi/lo (128-row boxes, the SM-pair kernel)
    alignas(64) unsigned char tmaps[6][128];
    alignas(64) unsigned char tmaps_y[6][128];  // the same with the targets' staging as A
    bool gemm_pair;       // projection GEMM on SM pairs (cta_group::2)
    // qs_sum's fork: the targets' operand split runs on side_st during the sources' GEMM;
    // sev = fork, join (no timing), split start, split end (timing, read by qs_stage_times)
    cudaStream_t side_st;
    cudaEvent_t sev[4];
    bool split_y_overlapped;  // the last timed qs_sum split the targets on side_st
    // stage timing (qs_set_timing)
    int timing;
    int timed_calls;
    cudaEvent_t ev[8];  // QS_NUM_STAGES + 1
    // qs_sum_host pipeline: copy stream and per-chunk arrival events (created by the first call)
    cudaStream_t copy_st;
    cudaEvent_t hev[1 + 2 * QS_HOST_CHUNKS];
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Tap values and first cell of a point at grid coordinate u.
//   l0 = ceil(u - m),  s = u - l0 - (m - 1/2) in (-1/2, 1/2]
//   tap[j] = psi(u - (l0 + j)),  j = 0 .. W-1
template <int W>
__device__ __forceinline__ void qs_taps(float u, const qs_window& win, int& l0, float (&tap)[W])
{
    constexpr int m = W / 2;
    constexpr int T = qs_tap_terms(W);
    const float fl = ceilf(u - (float)m);
    l0 = (int)fl;
    const float s = (u - fl) - ((float)m - 0.5f);
    const float s2 = s * s;
#pragma unroll
    for (int j = 0; j < m; ++j) {
        float e = win.e[j][T - 1];
        float o = win.o[j][T - 1];
#pragma unroll
        for (int i = T - 2; i >= 0; --i) {
            e = fmaf(e, s2, win.e[j][i]);
            o = fmaf(o, s2, win.o[j][i]);
        }
        tap[j] = fmaf(s, o, e);
        tap[W - 1 - j] = fmaf(-s, o, e);
    }
}

// Error-free transformation of a + b (Knuth's TwoSum); the rounding error is
// accumulated into lo.  No multiplications, so FMA contraction cannot alter it.
__device__ __forceinline__ void qs_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

// Two lanes of qs_two_sum in packed FP32x2 arithmetic (each lane rounds
// exactly as the scalar form; a - b is formed as fma(b, -1, a), the same
// correctly rounded difference).
__device__ __forceinline__ float2 qs_sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

__device__ __forceinline__ void qs_two_sum2(float2& hi, float2& lo, float2 x)
{
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = qs_sub2(s, hi);
    const float2 err = __fadd2_rn(qs_sub2(hi, qs_sub2(s, bp)), qs_sub2(x, bp));
    hi = s;
    lo = __fadd2_rn(lo, err);
}

// Validate a grid coordinate; returns a safe value and records the error.
__device__ __forceinline__ float qs_check_u(float u, float half_G, unsigned int* flag)
{
    if (!(fabsf(u) <= half_G)) {
        atomicOr(flag, (u != u || isinf(u)) ? QS_FLAG_NONFINITE : QS_FLAG_RANGE);
        return 0.0f;
    }
    return u;
}

// Targets per thread of the interpolation kernel (256 threads per CTA).
// Unfused: 8 (the per-slice staging and range work spread over more targets;
// measured faster than 4 at G = 2048 and G = 4096).
__host__ __device__ inline int qs_interp_tpt(bool fused, int d, int G)
{
    (void)G;
    return !fused ? 8 : (d <= 8 ? 2 : 1);
}

// ---------------------------------------------------------------------------
// host tables (qs_tables.cu): fixed-size outputs, no heap
// ---------------------------------------------------------------------------
double qs_tau_rule(qs_kernel kernel, double kparam, double R);
void qs_gauss_legendre(int n, double* x, double* w);
void qs_fit_window(int W, int kind, qs_window* win);
void qs_fill_atab(const qs_window* win, int W, float* atab);
double qs_window_tap(const qs_window* win, int W, int j, double s);
void qs_window_transform(const qs_window* win, int W, int K, int G, double* out);  // out[K + 1]
void qs_twiddles(int G, float2* out);                                               // out[G / 2]
// Sobol' points (qs_sobol.cu): u in (0,1)^d (P x d) and the unit rows Phi^{-1}(u) / |Phi^{-1}(u)|
qs_status qs_sobol_cube(int d, int P, uint64_t seed, double* out);
qs_status qs_sobol_sphere(int d, int P, uint64_t seed, float* out);
// autotune cache (qs_tune.cu): tuned spread variant / SM-pair GEMM choice (-1 = not tuned) of
// the plan's shape class (d bucket, N_ft, P bucket, projection form, W)
struct qs_plan_s;
bool qs_tune_lookup(const qs_plan_s* p, int* spread_variant, int* gemm_pair);
void qs_tune_store(const qs_plan_s* p, int spread_variant, int gemm_pair);

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files); return cudaSuccess or the launch error
// ---------------------------------------------------------------------------
int qs_sort_chunk(int P);
size_t qs_sort_workspace_bytes(int P, int64_t max_n, int64_t max_m);
cudaError_t qs_launch_sum_sorted(const float* x, int64_t N, const float* w, const float* y, int64_t M,
                                 const float* xi_s, const float* xi, int d, int P, double amp, void* ws,
                                 int64_t max_n, int64_t max_m, float* s, const float* v, float scale, float* gy,
                                 unsigned int* flag, cudaStream_t st);
cudaError_t qs_launch_coeffs(int kernel, double kparam, double kparam2, int d, double tau, int n_ft, int G,
                             const double* psihat, const double* c_in, double* c_out, float* D_out, cudaStream_t st);
cudaError_t qs_launch_project_fp32(const float* X, int64_t N, int d, const float* xi_s, int P,
                                   float* U, int64_t ldU, cudaStream_t st);
void qs_set_error_message(const char* msg);
cudaError_t qs_launch_deriv_table(const double* c, const double* psihat, int n_ft, int G, float* Dd, cudaStream_t st);
cudaError_t qs_launch_spread_grad(const qs_launch& L, int W, const float* x, const float* w, int mode, bool fused,
                                  const float* Dd, float* H2, cudaStream_t st);
cudaError_t qs_launch_interp_grad(const qs_launch& L, int W, const float* y, const float* Hd, const float* xi,
                                  float* part, bool fused, cudaStream_t st);
cudaError_t qs_launch_reduce_grad(const float* part, int S, int64_t M, int d, float scale, const float* fac,
                                  float* out, cudaStream_t st);
// unfused forms: derivative interpolation written over L.U (targets [0, L.M)), then
// out[m][j] = scale fac_m sum_p Q[p][m] xi[p][j]
cudaError_t qs_launch_interp_deriv(const qs_launch& L, int W, const float* Hd, cudaStream_t st);
cudaError_t qs_launch_backproj(const float* Q, int64_t ldQ, int64_t M, int P, const float* xi, int d, float scale,
                               const float* fac, float* out, cudaStream_t st);
bool qs_make_tmap(void* map_out, const void* base, int elem_bytes, int d, int64_t rows, int ldk, int box_rows);
// max_blocks > 0 caps the grid (a split running beside another kernel).
cudaError_t qs_launch_split_bf16(const float* X, int64_t rows, int d, int ldk, void* hi, void* lo, cudaStream_t st,
                                 int max_blocks = 0);
cudaError_t qs_launch_round_tf32(const float* X, int64_t rows, int d, int ldk, float* out, cudaStream_t st,
                                 int max_blocks = 0);
// Rows [n_base, n_base + N) of the staged operands into columns [n_base, n_base + N) of U;
// n_base a multiple of 128.
// pair: the SM-pair (cta_group::2) kernel, which needs maps 4 / 5 and qs_tc_pair_available.
cudaError_t qs_launch_project_tc(int kind, const void* maps, int64_t n_base, int64_t N, int d, int P, float* U,
                                 int64_t ldU, unsigned int* flag, cudaStream_t st, bool pair);
bool qs_tc_pair_available(int kind);
int qs_tc_pair_ctas(int kind);  // CTAs of a full-size SM-pair launch (2 x resident clusters)
cudaError_t qs_launch_weight_scale(const qs_launch& L, const float* w, cudaStream_t st);
cudaError_t qs_launch_spread(const qs_launch& L, int W, const float* x, const float* w, bool fused,
                             cudaStream_t st);
cudaError_t qs_launch_interp(const qs_launch& L, int W, const float* y, bool fused, cudaStream_t st);
cudaError_t qs_launch_reduce(const qs_launch& L, float* s, cudaStream_t st);
