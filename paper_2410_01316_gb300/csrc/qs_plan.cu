// Host side of the qmcslice C ABI: plans, directions, window tables and the
// orchestration of the sum pipeline (arXiv 2410.01316, App. C / App. G).
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "qs_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

thread_local char g_last_error[512] = "";

qs_status fail(qs_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

qs_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(QS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------
// seeded host random numbers: splitmix64 stream -> uniform (0,1) -> Box-Muller
// ---------------------------------------------------------------------------
struct HostRng {
    uint64_t state;
    explicit HostRng(uint64_t seed) : state(seed ^ 0x6a09e667f3bcc909ULL) {}
    uint64_t next()
    {
        uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u1 = uniform(), u2 = uniform();
        return sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2);
    }
};

// Haar-distributed d x d orthogonal matrix (column-major in q): Householder
// QR of a Gaussian matrix, with column i multiplied by sign(R_ii).
void haar_orthogonal(HostRng& rng, int d, std::vector<double>& q)
{
    std::vector<double> a((size_t)d * d);
    for (auto& v : a) v = rng.normal();  // a[i + j*d] = A(i, j)
    std::vector<double> vs((size_t)d * d, 0.0), rdiag(d);
    for (int k = 0; k < d; ++k) {
        double nrm = 0.0;
        for (int i = k; i < d; ++i) nrm += a[i + (size_t)k * d] * a[i + (size_t)k * d];
        nrm = sqrt(nrm);
        const double akk = a[k + (size_t)k * d];
        const double alpha = akk > 0 ? -nrm : nrm;  // R_kk
        rdiag[k] = alpha;
        double* v = &vs[(size_t)k * d];
        for (int i = 0; i < d; ++i) v[i] = 0.0;
        for (int i = k; i < d; ++i) v[i] = a[i + (size_t)k * d];
        v[k] -= alpha;
        double vn = 0.0;
        for (int i = k; i < d; ++i) vn += v[i] * v[i];
        if (vn > 0.0) {
            const double inv = 1.0 / sqrt(vn);
            for (int i = k; i < d; ++i) v[i] *= inv;
            for (int j = k; j < d; ++j) {  // A <- (I - 2 v v^T) A
                double dot = 0.0;
                for (int i = k; i < d; ++i) dot += v[i] * a[i + (size_t)j * d];
                for (int i = k; i < d; ++i) a[i + (size_t)j * d] -= 2.0 * dot * v[i];
            }
        }
    }
    // Q = H_0 H_1 ... H_{d-1}, accumulated backwards on the identity
    q.assign((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i) q[i + (size_t)i * d] = 1.0;
    for (int k = d - 1; k >= 0; --k) {
        const double* v = &vs[(size_t)k * d];
        for (int j = 0; j < d; ++j) {
            double dot = 0.0;
            for (int i = k; i < d; ++i) dot += v[i] * q[i + (size_t)j * d];
            for (int i = k; i < d; ++i) q[i + (size_t)j * d] -= 2.0 * dot * v[i];
        }
    }
    for (int j = 0; j < d; ++j) {
        const double sg = rdiag[j] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < d; ++i) q[i + (size_t)j * d] *= sg;
    }
}

// Fourier coefficients of the 1-periodic g(t) = f(|t| / tau), t in [-1/2, 1/2),
// for the generalised Riesz kernel (f = -c_{d,q} |t|^q, c_{d,q} =
// sqrt(pi) Gamma((d+q)/2) / (Gamma(d/2) Gamma((q+1)/2))) and the thin plate
// spline (f = d t^2 log|t| + C_d t^2, C_d = d/2 (H_{d/2} - 2 + log 4)), both
// from Table tab:kernels: c_k = 2 int_0^{1/2} g(t) cos(2 pi k t) dt for
// k = 0 .. n_ft/2, in FP64.  All k share one set of nodes: 16-point
// Gauss-Legendre on panels of width 1/n_ft (half a period of the highest
// frequency), the first panel split geometrically towards t = 0 where g is
// not smooth; cos(2 pi k t) over k by the three-term recurrence, restarted
// from cos() every 64 steps.  Writes c[k + n_ft/2] for k = -n_ft/2 .. n_ft/2 - 1.
void periodic_coeffs(qs_kernel kernel, double q, int d, double tau, int n_ft, std::vector<double>& c)
{
    const int K = n_ft / 2;
    double amp = 0.0, cd = 0.0;
    if (kernel == QS_RIESZ) {
        amp = -exp(0.5 * log(kPi) + lgamma(0.5 * (d + q)) - lgamma(0.5 * d) - lgamma(0.5 * (q + 1.0)));
    } else {
        double h = 0.0, x = 0.0;  // H_x at x = 0 or 1/2, stepped up to d/2
        if (d & 1) {
            h = 2.0 - 2.0 * log(2.0);
            x = 0.5;
        }
        for (; x + 0.25 < 0.5 * d; x += 1.0) h += 1.0 / (x + 1.0);
        cd = 0.5 * d * (h - 2.0 + log(4.0));
    }
    auto g = [&](double t) {
        const double u = t / tau;
        if (kernel == QS_RIESZ) return amp * pow(u, q);
        return u > 0.0 ? (double)d * u * u * log(u) + cd * u * u : 0.0;
    };
    constexpr int nq = 16;
    double gx[nq], gw[nq];
    qs_gauss_legendre(nq, gx, gw);
    std::vector<double> nodes, vals;
    auto panel = [&](double a, double b) {
        const double m = 0.5 * (a + b), hh = 0.5 * (b - a);
        for (int i = 0; i < nq; ++i) {
            const double t = m + hh * gx[i];
            nodes.push_back(t);
            vals.push_back(2.0 * hh * gw[i] * g(t));
        }
    };
    const double h = 0.5 / K;
    for (int j = 1; j < K; ++j) panel(j * h, (j + 1) * h);
    for (double b = h; b > h * 1e-18; b *= 0.5) panel(0.5 * b, b);
    std::vector<double> acc(K + 1, 0.0);
    for (size_t i = 0; i < nodes.size(); ++i) {
        const double th = 2.0 * kPi * nodes[i], c1 = cos(th), v = vals[i];
        acc[0] += v;
        acc[1] += v * c1;
        double cprev = 1.0, ccur = c1;  // cos((k-2) th), cos((k-1) th)
        for (int k = 2; k <= K; ++k) {
            double cnext;
            if ((k & 63) == 0) {
                ccur = cos((k - 1) * th);
                cnext = cos(k * th);
            } else {
                cnext = 2.0 * c1 * ccur - cprev;
            }
            acc[k] += v * cnext;
            cprev = ccur;
            ccur = cnext;
        }
    }
    c.assign(n_ft, 0.0);
    for (int k = 0; k <= K; ++k) {
        if (k < K) c[K + k] = acc[k];
        c[K - k] = acc[k];
    }
}

void free_plan(qs_plan p)
{
    if (!p) return;
    for (int i = 0; i < QS_NUM_STAGES + 1; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    for (int i = 0; i < 1 + 2 * QS_HOST_CHUNKS; ++i)
        if (p->hev[i]) cudaEventDestroy(p->hev[i]);
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
    for (int i = 0; i < 4; ++i)
        if (p->sev[i]) cudaEventDestroy(p->sev[i]);
    if (p->side_st) cudaStreamDestroy(p->side_st);
    void* bufs[] = {p->d_dirs, p->d_dirs_s, p->d_c, p->d_psihat, p->d_D, p->d_tw, p->d_U, p->d_H,
                    p->d_part, p->d_flag, p->d_wscale, p->d_x, p->d_w, p->d_y, p->d_s, p->d_xi_hi, p->d_xi_lo,
                    p->d_xs_hi, p->d_xs_lo, p->d_ys_hi, p->d_ys_lo, p->d_Dd, p->d_H2, p->d_gpart, p->d_sortws};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete p;
}

template <class T>
cudaError_t dalloc(T** ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)ptr, count * sizeof(T));
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// targets_per_cta: targets covered by one CTA of the interpolation kernel that
// will consume the launch (256 x targets per thread; 256 for the gradients).
qs_launch make_launch(const qs_plan p, int64_t N, int64_t M, int64_t targets_per_cta)
{
    qs_launch L;
    memset(&L, 0, sizeof(L));
    L.d = p->desc.d;
    L.P = p->desc.P;
    L.G = p->G;
    L.n_ft = p->desc.n_ft;
    L.N = N;
    L.M = M;
    L.m_base = 0;
    L.m_end = M;
    L.ldU = p->ldU;
    L.half_G = 0.5f * (float)p->G;
    L.xi_s = p->d_dirs_s;
    L.D = p->d_D;
    L.tw = p->d_tw;
    L.H = p->d_H;
    L.U = p->d_U;
    L.part = p->d_part;
    L.flag = p->d_flag;
    L.wscale = p->d_wscale;
    L.spread_variant = p->spread_variant;
    L.win = p->win;
    qs_fill_atab(&p->win, p->W, L.atab);
    // slice groups of the interpolation: enough CTAs to fill the device,
    // chosen from M and P only so results do not depend on the GPU model
    const int64_t blocks_m = (M + targets_per_cta - 1) / targets_per_cta;
    int64_t S = (1024 + blocks_m - 1) / (blocks_m > 0 ? blocks_m : 1);
    if (S < 1) S = 1;
    if (S > p->S_max) S = p->S_max;
    L.S = (int)S;
    return L;
}

// Operand preparation of the tensor-core forms (BF16 hi/lo split or TF32
// rounding of the points into the plan's staging: the targets' own staging
// when ystage, so that it can run while the sources' GEMM reads theirs);
// nothing for FP32.
cudaError_t project_prep(const qs_plan p, const float* X, int64_t rows, cudaStream_t st, bool ystage = false)
{
    const int d = p->desc.d;
    void* hi = ystage ? p->d_ys_hi : p->d_xs_hi;
    void* lo = ystage ? p->d_ys_lo : p->d_xs_lo;
    // the targets' split runs beside the sources' GEMM: two blocks per SM
    // leave the GEMM's epilogue warps their issue slots and still move the
    // operands well within the GEMM's duration
    const int cap = ystage ? 2 * p->sm_count : 0;
    switch (p->proj) {
        case QS_PROJ_BF16X3: return qs_launch_split_bf16(X, rows, d, p->ldk, hi, lo, st, cap);
        case QS_PROJ_TF32: return qs_launch_round_tf32(X, rows, d, p->ldk, (float*)hi, st, cap);
        default: return cudaSuccess;
    }
}

// The projection GEMM U = G tau X Xi^T (after project_prep for the tensor-core forms).
cudaError_t project_gemm(const qs_plan p, const float* X, int64_t rows, cudaStream_t st, bool ystage = false)
{
    const int d = p->desc.d, P = p->desc.P;
    const void* maps = ystage ? (const void*)p->tmaps_y : (const void*)p->tmaps;
    switch (p->proj) {
        case QS_PROJ_FP32: return qs_launch_project_fp32(X, rows, d, p->d_dirs_s, P, p->d_U, p->ldU, st);
        case QS_PROJ_BF16X3:
            return qs_launch_project_tc(0, maps, 0, rows, d, P, p->d_U, p->ldU, p->d_flag, st, p->gemm_pair);
        case QS_PROJ_TF32:
            return qs_launch_project_tc(1, maps, 0, rows, d, P, p->d_U, p->ldU, p->d_flag, st, p->gemm_pair);
        default: return cudaErrorInvalidValue;
    }
}

// Rows [r0, r0 + rows) of X (N x d, row-major) projected into columns
// [r0, r0 + rows) of U, operand preparation included; r0 a multiple of 128.
cudaError_t project_rows(const qs_plan p, const float* X, int64_t r0, int64_t rows, cudaStream_t st)
{
    const int d = p->desc.d, P = p->desc.P;
    const float* Xr = X + r0 * d;
    cudaError_t e;
    switch (p->proj) {
        case QS_PROJ_FP32: return qs_launch_project_fp32(Xr, rows, d, p->d_dirs_s, P, p->d_U + r0, p->ldU, st);
        case QS_PROJ_BF16X3:
            e = qs_launch_split_bf16(Xr, rows, d, p->ldk, (uint16_t*)p->d_xs_hi + r0 * p->ldk,
                                     (uint16_t*)p->d_xs_lo + r0 * p->ldk, st);
            return e == cudaSuccess ? qs_launch_project_tc(0, p->tmaps, r0, rows, d, P, p->d_U, p->ldU, p->d_flag, st,
                                                           p->gemm_pair)
                                    : e;
        case QS_PROJ_TF32:
            e = qs_launch_round_tf32(Xr, rows, d, p->ldk, (float*)p->d_xs_hi + r0 * p->ldk, st);
            return e == cudaSuccess ? qs_launch_project_tc(1, p->tmaps, r0, rows, d, P, p->d_U, p->ldU, p->d_flag, st,
                                                           p->gemm_pair)
                                    : e;
        default: return cudaErrorInvalidValue;
    }
}

// Rows per chunk of the qs_sum_host pipeline: at most `chunks` chunks, a
// multiple of `unit` (a multiple of the GEMM's 128-row tile), at least 4096 rows.
int64_t host_chunk_rows(int64_t n, int64_t unit = 128, int chunks = QS_HOST_CHUNKS)
{
    int64_t c = (n + chunks - 1) / chunks;
    c = (c + unit - 1) / unit * unit;
    return c < 4096 ? (4096 + unit - 1) / unit * unit : c;
}

// U = G tau X Xi^T for the plan's projection form.
cudaError_t project(const qs_plan p, const float* X, int64_t rows, cudaStream_t st)
{
    cudaError_t e = project_prep(p, X, rows, st);
    return e == cudaSuccess ? project_gemm(p, X, rows, st) : e;
}

}  // namespace

// Set the thread's last-error message (for entry points defined in other files).
void qs_set_error_message(const char* msg)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg ? msg : "");
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* qs_version(void) { return "qmcslice 0.1 (sm_103a)"; }

const char* qs_last_error(void) { return g_last_error; }

const char* qs_status_string(qs_status s)
{
    switch (s) {
        case QS_OK: return "ok";
        case QS_ERR_ARG: return "invalid argument";
        case QS_ERR_RANGE: return "projection outside the half period (radius too small)";
        case QS_ERR_NONFINITE: return "non-finite input value";
        case QS_ERR_OOM: return "out of memory";
        case QS_ERR_CUDA: return "CUDA runtime error";
        case QS_ERR_UNSUPPORTED: return "unsupported configuration";
        case QS_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

qs_status qs_directions(qs_dirs kind, int d, int P, uint64_t seed, float* out)
{
    if (!out || d < 1 || P < 1) return fail(QS_ERR_ARG, "qs_directions: bad arguments");
    if (kind == QS_DIR_FIBONACCI) {
        if (d != 3) return fail(QS_ERR_ARG, "qs_directions: Fibonacci directions need d = 3");
        const double golden = 0.5 * (1.0 + sqrt(5.0));
        for (int p = 0; p < P; ++p) {
            const double z = 1.0 - (2.0 * p + 1.0) / P;
            const double phi = 2.0 * kPi * p / golden;
            const double r = sqrt(fmax(0.0, 1.0 - z * z));
            out[3 * p + 0] = (float)(r * cos(phi));
            out[3 * p + 1] = (float)(r * sin(phi));
            out[3 * p + 2] = (float)z;
        }
        return QS_OK;
    }
    HostRng rng(seed);
    if (kind == QS_DIR_IID) {
        std::vector<double> g(d);
        for (int p = 0; p < P; ++p) {
            double nrm = 0.0;
            for (int j = 0; j < d; ++j) {
                g[j] = rng.normal();
                nrm += g[j] * g[j];
            }
            nrm = sqrt(nrm);
            for (int j = 0; j < d; ++j) out[(size_t)p * d + j] = (float)(g[j] / nrm);
        }
        return QS_OK;
    }
    if (kind == QS_DIR_ORTHOGONAL) {
        std::vector<double> q;
        for (int p0 = 0; p0 < P; p0 += d) {
            haar_orthogonal(rng, d, q);
            for (int c = 0; c < d && p0 + c < P; ++c)
                for (int j = 0; j < d; ++j) out[(size_t)(p0 + c) * d + j] = (float)q[j + (size_t)c * d];
        }
        return QS_OK;
    }
    if (kind == QS_DIR_SOBOL) {
        if (d > QS_SOBOL_MAX_D) return fail(QS_ERR_UNSUPPORTED, "qs_directions: Sobol' directions need d <= %d",
                                            QS_SOBOL_MAX_D);
        const qs_status st = qs_sobol_sphere(d, P, seed, out);
        return st == QS_OK ? QS_OK : fail(st, "qs_directions: Sobol' directions unavailable for d = %d", d);
    }
    if (kind == QS_DIR_DISTANCE)
        return fail(QS_ERR_UNSUPPORTED, "qs_directions: distance designs are optimised on the GPU "
                                        "(QS_DIR_DISTANCE in a plan, or qs_distance_design)");
    return fail(QS_ERR_ARG, "qs_directions: unknown kind %d", (int)kind);
}

qs_status qs_plan_create(qs_plan* out, const qs_plan_desc* desc)
{
    if (!out || !desc) return fail(QS_ERR_ARG, "qs_plan_create: NULL argument");
    *out = nullptr;
    const qs_plan_desc& D = *desc;
    if (D.d < 1 || D.P < 1) return fail(QS_ERR_ARG, "qs_plan_create: d and P must be >= 1");
    if (D.kernel < QS_GAUSS || D.kernel > QS_TPS)
        return fail(QS_ERR_ARG, "qs_plan_create: unknown kernel %d", (int)D.kernel);
    if ((D.kernel == QS_GAUSS || D.kernel == QS_LAPLACE || D.kernel == QS_MATERN) &&
        !(D.kparam > 0.0 && isfinite(D.kparam)))
        return fail(QS_ERR_ARG, "qs_plan_create: kernel parameter must be positive");
    if (D.kernel == QS_MATERN && !(D.kparam2 > 0.0 && D.kparam2 < 1e6))
        return fail(QS_ERR_ARG, "qs_plan_create: Matern nu (kparam2) must be positive");
    if (D.kernel == QS_RIESZ && !(D.kparam > 0.0 && D.kparam < 2.0))
        return fail(QS_ERR_ARG, "qs_plan_create: Riesz exponent (kparam) must lie in (0, 2)");
    if (!(D.radius > 0.0 && isfinite(D.radius))) return fail(QS_ERR_ARG, "qs_plan_create: radius must be > 0");
    if (!is_pow2(D.n_ft) || D.n_ft < 16 || D.n_ft > QS_MAX_G / 2)
        return fail(QS_ERR_UNSUPPORTED, "qs_plan_create: n_ft must be a power of two in [16, %d]", QS_MAX_G / 2);
    const int W = D.window == 0 ? 8 : D.window;
    if (W != 6 && W != 8 && W != 10 && W != 12)
        return fail(QS_ERR_UNSUPPORTED, "qs_plan_create: window must be 6, 8, 10 or 12");
    if (D.window_kind != QS_WINDOW_ES && D.window_kind != QS_WINDOW_KB)
        return fail(QS_ERR_ARG, "qs_plan_create: unknown window kind %d", (int)D.window_kind);
    const double os = D.oversampling == 0.0 ? 2.0 : D.oversampling;
    if (os != 2.0) return fail(QS_ERR_UNSUPPORTED, "qs_plan_create: only oversampling 2 is supported");
    if (D.max_n < 0 || D.max_m < 0) return fail(QS_ERR_ARG, "qs_plan_create: max_n / max_m must be >= 0");
    if (D.dirs == QS_DIR_USER && !D.dirs_host) return fail(QS_ERR_ARG, "qs_plan_create: dirs_host is NULL");
    if (D.dirs < QS_DIR_USER || D.dirs > QS_DIR_SOBOL)
        return fail(QS_ERR_ARG, "qs_plan_create: unknown direction kind %d", (int)D.dirs);
    if (D.dirs == QS_DIR_FIBONACCI && D.d != 3)
        return fail(QS_ERR_ARG, "qs_plan_create: Fibonacci directions need d = 3");

    // AUTO: the fused form re-reads d coordinates per point and slice with a
    // strided pattern and only pays off for very small d; the SIMT GEMM is
    // cheapest below d = 64 and the BF16x3 tensor-core GEMM from there on
    qs_proj proj = D.proj;
    if (proj == QS_PROJ_AUTO) proj = D.d <= 4 ? QS_PROJ_FP32_FUSED : (D.d < 64 ? QS_PROJ_FP32 : QS_PROJ_BF16X3);
    if (proj == QS_PROJ_FP32_FUSED && D.d > QS_FUSED_MAX_D)
        return fail(QS_ERR_UNSUPPORTED, "qs_plan_create: fused projection needs d <= %d", QS_FUSED_MAX_D);
    if (proj != QS_PROJ_FP32 && proj != QS_PROJ_FP32_FUSED && proj != QS_PROJ_BF16X3 && proj != QS_PROJ_TF32)
        return fail(QS_ERR_UNSUPPORTED, "qs_plan_create: projection form %d not available", (int)proj);

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "qs_plan_create: cudaGetDevice");
    int sms = 0;
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "qs_plan_create: device attribute");

    qs_plan p = new (std::nothrow) qs_plan_s;
    if (!p) return fail(QS_ERR_OOM, "qs_plan_create: host allocation");
    memset(p, 0, sizeof(*p));
    p->device = dev;
    p->sm_count = sms;
    p->desc = D;
    p->desc.dirs_host = nullptr;
    p->desc.window = W;
    p->desc.oversampling = os;
    p->proj = proj;
    p->W = W;
    p->G = 2 * D.n_ft;
    p->spread_variant = qs_spread_default(p->G, W);
    p->window_kind = D.window_kind;
    p->tau = qs_tau_rule(D.kernel, D.kparam, D.radius);
    p->S_max = D.P < 64 ? D.P : 64;
    const int64_t maxnm = D.max_n > D.max_m ? D.max_n : D.max_m;
    p->ldU = ((maxnm + 127) / 128) * 128;
    if (p->ldU == 0) p->ldU = 128;
    const int G = p->G, K = D.n_ft / 2, d = D.d, P = D.P;

    // directions (host), FP32
    std::vector<float> dirs((size_t)P * d);
    if (D.dirs == QS_DIR_USER) {
        for (size_t i = 0; i < dirs.size(); ++i) {
            if (!isfinite(desc->dirs_host[i])) {
                free_plan(p);
                return fail(QS_ERR_ARG, "qs_plan_create: non-finite direction entry");
            }
            dirs[i] = desc->dirs_host[i];
        }
    } else {
        const bool distance = D.dirs == QS_DIR_DISTANCE;
        qs_status st = qs_directions(distance ? QS_DIR_ORTHOGONAL : D.dirs, d, P, D.seed, dirs.data());
        if (st == QS_OK && distance) {
            // refine the seeded orthogonal start into a distance design on the device
            float* d_tmp = nullptr;
            const size_t bytes = dirs.size() * sizeof(float);
            if (cudaMalloc(&d_tmp, bytes) != cudaSuccess) {
                st = QS_ERR_OOM;
            } else {
                if (cudaMemcpy(d_tmp, dirs.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) st = QS_ERR_CUDA;
                if (st == QS_OK) st = qs_distance_design(d_tmp, d, P, 300, 0.05 / sqrt((double)d), nullptr, nullptr);
                if (st == QS_OK && cudaMemcpy(dirs.data(), d_tmp, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
                    st = QS_ERR_CUDA;
                cudaFree(d_tmp);
            }
        }
        if (st != QS_OK) {
            free_plan(p);
            return st;
        }
    }
    std::vector<float> dirs_s(dirs.size());
    const double scale = (double)G * p->tau;
    for (size_t i = 0; i < dirs.size(); ++i) dirs_s[i] = (float)(scale * (double)dirs[i]);

    // window tables
    qs_fit_window(W, p->window_kind, &p->win);
    std::vector<double> psihat(K + 1);
    qs_window_transform(&p->win, W, K, G, psihat.data());
    std::vector<float2> tw(G / 2);
    qs_twiddles(G, tw.data());

    // device buffers
#define QS_ALLOC(ptr, n)                                                       \
    do {                                                                       \
        cudaError_t e_ = dalloc(&(ptr), (n));                                  \
        if (e_ != cudaSuccess) {                                               \
            cudaGetLastError();                                                \
            free_plan(p);                                                      \
            return fail(QS_ERR_OOM, "qs_plan_create: cudaMalloc(%s, %zu B): %s", #ptr, \
                        (size_t)(n) * sizeof(*(ptr)), cudaGetErrorString(e_)); \
        }                                                                      \
    } while (0)
    QS_ALLOC(p->d_dirs, (size_t)P * d);
    QS_ALLOC(p->d_dirs_s, (size_t)P * d);
    QS_ALLOC(p->d_c, (size_t)D.n_ft);
    QS_ALLOC(p->d_psihat, (size_t)K + 1);
    QS_ALLOC(p->d_D, (size_t)G / 2 + 1);
    QS_ALLOC(p->d_tw, (size_t)G / 2);
    QS_ALLOC(p->d_H, (size_t)P * G);
    // slice-group partials: sized for targets up to max(max_n, max_m), since the
    // gradients evaluate at x as well as at y
    QS_ALLOC(p->d_part, (size_t)2 * p->S_max * (maxnm > 0 ? maxnm : 1));
    if (d <= QS_GRAD_MAX_D && proj == QS_PROJ_FP32_FUSED) {
        // per-component gradient partials of the fused form (the unfused forms
        // back-project with a GEMM): largest S(M) * M over M <= max(max_n, max_m), S as in make_launch
        size_t sm = 1;
        for (int64_t b = 1; b <= (maxnm + 255) / 256; ++b) {
            int64_t S = (1024 + b - 1) / b;
            if (S > p->S_max) S = p->S_max;
            const int64_t rows = 256 * b < maxnm ? 256 * b : maxnm;
            if ((size_t)(S * rows) > sm) sm = (size_t)(S * rows);
        }
        p->gpart_elems = 2 * sm * (size_t)d;
        QS_ALLOC(p->d_gpart, p->gpart_elems);
    }
    if (d <= QS_GRAD_MAX_D || proj != QS_PROJ_FP32_FUSED) {
        // derivative filter and grid (the unfused forms back-project with a GEMM
        // from the projection buffer, the fused form with d per-component partials)
        QS_ALLOC(p->d_Dd, (size_t)G / 2 + 1);
        QS_ALLOC(p->d_H2, (size_t)P * G);
    }
    QS_ALLOC(p->d_flag, 1);
    QS_ALLOC(p->d_wscale, 2);
    const bool tc = proj == QS_PROJ_BF16X3 || proj == QS_PROJ_TF32;
    if (proj == QS_PROJ_FP32 || tc) {
        p->U_elems = (size_t)P * (size_t)p->ldU;
        QS_ALLOC(p->d_U, p->U_elems);
    }
    const int64_t stage_rows = maxnm > 0 ? maxnm : 1;
    const int64_t ystage_rows = D.max_m > 0 ? D.max_m : 1;
    if (proj == QS_PROJ_BF16X3) {
        p->ldk = (d + 7) / 8 * 8;  // 16-byte row stride for TMA
        uint16_t *xh = nullptr, *xl = nullptr, *sh = nullptr, *sl = nullptr;
        QS_ALLOC(xh, (size_t)P * p->ldk);
        p->d_xi_hi = xh;
        QS_ALLOC(xl, (size_t)P * p->ldk);
        p->d_xi_lo = xl;
        QS_ALLOC(sh, (size_t)stage_rows * p->ldk);
        p->d_xs_hi = sh;
        QS_ALLOC(sl, (size_t)stage_rows * p->ldk);
        p->d_xs_lo = sl;
        uint16_t *yh = nullptr, *yl = nullptr;
        QS_ALLOC(yh, (size_t)ystage_rows * p->ldk);
        p->d_ys_hi = yh;
        QS_ALLOC(yl, (size_t)ystage_rows * p->ldk);
        p->d_ys_lo = yl;
    } else if (proj == QS_PROJ_TF32) {
        p->ldk = (d + 3) / 4 * 4;
        float *xh = nullptr, *sh = nullptr, *yh = nullptr;
        QS_ALLOC(xh, (size_t)P * p->ldk);
        p->d_xi_hi = xh;
        QS_ALLOC(sh, (size_t)stage_rows * p->ldk);
        p->d_xs_hi = sh;
        QS_ALLOC(yh, (size_t)ystage_rows * p->ldk);
        p->d_ys_hi = yh;
    }
    QS_ALLOC(p->d_x, (size_t)(D.max_n > 0 ? D.max_n : 1) * d);
    QS_ALLOC(p->d_w, (size_t)(D.max_n > 0 ? D.max_n : 1));
    QS_ALLOC(p->d_y, (size_t)(D.max_m > 0 ? D.max_m : 1) * d);
    QS_ALLOC(p->d_s, (size_t)(D.max_m > 0 ? D.max_m : 1));
#undef QS_ALLOC

#define QS_CHECK(call, what)          \
    do {                              \
        cudaError_t e_ = (call);      \
        if (e_ != cudaSuccess) {      \
            free_plan(p);             \
            return cuda_fail(e_, what); \
        }                             \
    } while (0)
    QS_CHECK(cudaMemcpy(p->d_dirs, dirs.data(), dirs.size() * sizeof(float), cudaMemcpyHostToDevice), "copy dirs");
    QS_CHECK(cudaMemcpy(p->d_dirs_s, dirs_s.data(), dirs_s.size() * sizeof(float), cudaMemcpyHostToDevice),
             "copy scaled dirs");
    QS_CHECK(cudaMemcpy(p->d_psihat, psihat.data(), psihat.size() * sizeof(double), cudaMemcpyHostToDevice),
             "copy window transform");
    QS_CHECK(cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice), "copy twiddles");
    QS_CHECK(cudaMemset(p->d_flag, 0, sizeof(unsigned int)), "clear flag");
    if (D.kernel == QS_RIESZ || D.kernel == QS_TPS) {
        // no classical transform: the periodised kernel's coefficients by host quadrature
        std::vector<double> ch;
        periodic_coeffs(D.kernel, D.kparam, d, p->tau, D.n_ft, ch);
        double* d_ch = nullptr;
        QS_CHECK(cudaMalloc(&d_ch, ch.size() * sizeof(double)), "coefficient table");
        cudaError_t e1 = cudaMemcpy(d_ch, ch.data(), ch.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e1 == cudaSuccess)
            e1 = qs_launch_coeffs((int)D.kernel, D.kparam, D.kparam2, d, p->tau, D.n_ft, G, p->d_psihat, d_ch,
                                  p->d_c, p->d_D, 0);
        if (e1 == cudaSuccess) e1 = cudaDeviceSynchronize();
        cudaFree(d_ch);
        QS_CHECK(e1, "coefficient table upload");
    } else {
        QS_CHECK(qs_launch_coeffs((int)D.kernel, D.kparam, D.kparam2, d, p->tau, D.n_ft, G, p->d_psihat, nullptr,
                                  p->d_c, p->d_D, 0),
                 "coefficient kernel launch");
    }
    if (p->d_Dd) QS_CHECK(qs_launch_deriv_table(p->d_c, p->d_psihat, D.n_ft, G, p->d_Dd, 0), "derivative table");
    if (tc) {
        const int eb = proj == QS_PROJ_BF16X3 ? 2 : 4;
        if (proj == QS_PROJ_BF16X3)
            QS_CHECK(qs_launch_split_bf16(p->d_dirs_s, P, d, p->ldk, p->d_xi_hi, p->d_xi_lo, 0), "split directions");
        else
            QS_CHECK(qs_launch_round_tf32(p->d_dirs_s, P, d, p->ldk, (float*)p->d_xi_hi, 0), "round directions");
        bool ok = qs_make_tmap(p->tmaps[0], p->d_xs_hi, eb, d, stage_rows, p->ldk, 128) &&
                  qs_make_tmap(p->tmaps[2], p->d_xi_hi, eb, d, P, p->ldk, 256) &&
                  qs_make_tmap(p->tmaps[4], p->d_xi_hi, eb, d, P, p->ldk, 128);
        if (ok && proj == QS_PROJ_BF16X3)
            ok = qs_make_tmap(p->tmaps[1], p->d_xs_lo, eb, d, stage_rows, p->ldk, 128) &&
                 qs_make_tmap(p->tmaps[3], p->d_xi_lo, eb, d, P, p->ldk, 256) &&
                 qs_make_tmap(p->tmaps[5], p->d_xi_lo, eb, d, P, p->ldk, 128);
        memcpy(p->tmaps_y, p->tmaps, sizeof(p->tmaps));
        if (ok) ok = qs_make_tmap(p->tmaps_y[0], p->d_ys_hi, eb, d, ystage_rows, p->ldk, 128);
        if (ok && proj == QS_PROJ_BF16X3) ok = qs_make_tmap(p->tmaps_y[1], p->d_ys_lo, eb, d, ystage_rows, p->ldk, 128);
        if (!ok) {
            free_plan(p);
            return fail(QS_ERR_CUDA, "qs_plan_create: cuTensorMapEncodeTiled failed");
        }
        QS_CHECK(cudaStreamCreateWithFlags(&p->side_st, cudaStreamNonBlocking), "side stream");
        for (int i = 0; i < 4; ++i)
            QS_CHECK(cudaEventCreateWithFlags(&p->sev[i], i < 2 ? cudaEventDisableTiming : cudaEventDefault),
                     "fork / join events");
        // the SM-pair GEMM where the GEMM is tensor-bound (d >= 256: 6 d flop
        // per 4 B of U written) and two-CTA clusters of it can be resident;
        // below, the U stores bound both forms and the single-SM one is faster
        // (d = 64: 0.80 against 0.93 ms for N = 2e5, P = 4096)
        p->gemm_pair = d >= 256 && qs_tc_pair_available(proj == QS_PROJ_BF16X3 ? 0 : 1);
    }
    QS_CHECK(cudaDeviceSynchronize(), "coefficient kernel");
#undef QS_CHECK
    // choices tuned earlier for this shape class (autotune cache)
    {
        int tv = -1, tp = -1;
        if (qs_tune_lookup(p, &tv, &tp)) {
            if (tv >= 0 && qs_spread_variant_ok(G, W, tv)) p->spread_variant = tv;
            if (tp >= 0 && tc && (tp == 0 || qs_tc_pair_available(proj == QS_PROJ_BF16X3 ? 0 : 1)))
                p->gemm_pair = tp == 1;
        }
    }
    *out = p;
    g_last_error[0] = 0;
    return QS_OK;
}

qs_status qs_plan_destroy(qs_plan p)
{
    if (!p) return QS_OK;
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    return QS_OK;
}

qs_status qs_plan_info(qs_plan p, double* tau, int* grid_size, int* P, const float** dirs_dev)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_info: NULL plan");
    if (tau) *tau = p->tau;
    if (grid_size) *grid_size = p->G;
    if (P) *P = p->desc.P;
    if (dirs_dev) *dirs_dev = p->d_dirs;
    return QS_OK;
}

qs_status qs_plan_directions(qs_plan p, float* dirs_host)
{
    if (!p || !dirs_host) return fail(QS_ERR_ARG, "qs_plan_directions: NULL argument");
    DeviceGuard g(p->device);
    cudaError_t e = cudaMemcpy(dirs_host, p->d_dirs, (size_t)p->desc.P * p->desc.d * sizeof(float),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qs_plan_directions");
    return QS_OK;
}

qs_status qs_sum(qs_plan p, const float* x, int64_t N, const float* w, const float* y, int64_t M, float* s,
                 void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_sum: NULL plan");
    if (N < 0 || M < 0) return fail(QS_ERR_ARG, "qs_sum: negative size");
    if (N > p->desc.max_n || M > p->desc.max_m)
        return fail(QS_ERR_ARG, "qs_sum: N=%lld / M=%lld exceed the plan's max_n=%lld / max_m=%lld",
                    (long long)N, (long long)M, (long long)p->desc.max_n, (long long)p->desc.max_m);
    if ((N > 0 && !x) || (M > 0 && (!y || !s))) return fail(QS_ERR_ARG, "qs_sum: NULL data pointer");
    if (M == 0) return QS_OK;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (N == 0) {
        e = cudaMemsetAsync(s, 0, (size_t)M * sizeof(float), st);
        return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_sum: memset");
    }
    const bool fused = p->proj == QS_PROJ_FP32_FUSED;
    qs_launch L = make_launch(p, N, M, 256 * qs_interp_tpt(fused, p->desc.d, p->G));
    const bool tm = p->timing != 0;
#define QS_MARK(i)                                              \
    do {                                                        \
        if (tm) {                                               \
            e = cudaEventRecord(p->ev[i], st);                  \
            if (e != cudaSuccess) return cuda_fail(e, "qs_sum: timing event"); \
        }                                                       \
    } while (0)
    QS_MARK(0);
    if (!fused) {
        e = project_prep(p, x, N, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: operand split of x");
    }
    QS_MARK(1);
    // tensor-core forms with d >= 256: the targets' operand split (HBM-bound)
    // runs on the side stream, in its own staging, while the sources' GEMM
    // runs (tensor-bound there: 6 d flop per 4 B of U written; below that the
    // GEMM is bound by its U stores and the split would slow it); the main
    // stream joins it before the targets' GEMM
    const bool fork = p->side_st != nullptr && (p->proj == QS_PROJ_BF16X3 || p->proj == QS_PROJ_TF32) &&
                      p->desc.d >= 256;
    if (fork) {
        e = cudaEventRecord(p->sev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side_st, p->sev[0], 0);
        if (e == cudaSuccess && tm) e = cudaEventRecord(p->sev[2], p->side_st);
        if (e == cudaSuccess) e = project_prep(p, y, M, p->side_st, true);
        if (e == cudaSuccess && tm) e = cudaEventRecord(p->sev[3], p->side_st);
        if (e == cudaSuccess) e = cudaEventRecord(p->sev[1], p->side_st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: operand split of y");
    }
    if (!fused) {
        e = project_gemm(p, x, N, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: projection of x");
    }
    QS_MARK(2);
    e = qs_launch_weight_scale(L, w, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sum: weight bound");
    e = qs_launch_spread(L, p->W, x, w, fused, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sum: spread");
    QS_MARK(3);
    if (fork) {
        e = cudaStreamWaitEvent(st, p->sev[1], 0);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: join");
    } else if (!fused) {
        e = project_prep(p, y, M, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: operand split of y");
    }
    QS_MARK(4);
    if (!fused) {
        e = project_gemm(p, y, M, st, fork);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum: projection of y");
    }
    QS_MARK(5);
    e = qs_launch_interp(L, p->W, y, fused, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sum: interpolation");
    QS_MARK(6);
    e = qs_launch_reduce(L, s, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sum: reduction");
    QS_MARK(7);
#undef QS_MARK
    if (tm) {
        p->timed_calls++;
        p->split_y_overlapped = fork;
    }
    return QS_OK;
}

qs_status qs_set_timing(qs_plan p, int enable)
{
    if (!p) return fail(QS_ERR_ARG, "qs_set_timing: NULL plan");
    DeviceGuard g(p->device);
    if (enable && !p->ev[0]) {
        for (int i = 0; i < QS_NUM_STAGES + 1; ++i) {
            cudaError_t e = cudaEventCreate(&p->ev[i]);
            if (e != cudaSuccess) return cuda_fail(e, "qs_set_timing: cudaEventCreate");
        }
    }
    p->timing = enable ? 1 : 0;
    p->timed_calls = 0;
    return QS_OK;
}

qs_status qs_stage_times(qs_plan p, float* ms, int n)
{
    if (!p || !ms || n < 0) return fail(QS_ERR_ARG, "qs_stage_times: bad argument");
    if (!p->ev[0] || p->timed_calls == 0) return fail(QS_ERR_ARG, "qs_stage_times: no timed call recorded");
    DeviceGuard g(p->device);
    cudaError_t e = cudaEventSynchronize(p->ev[QS_NUM_STAGES]);
    if (e != cudaSuccess) return cuda_fail(e, "qs_stage_times: event");
    for (int i = 0; i < n && i < QS_NUM_STAGES; ++i) {
        float t = 0.0f;
        if (i == 3 && p->split_y_overlapped)  // the side stream's split, run during the GEMM of x
            e = cudaEventElapsedTime(&t, p->sev[2], p->sev[3]);
        else
            e = cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "qs_stage_times: elapsed");
        ms[i] = t;
    }
    for (int i = QS_NUM_STAGES; i < n; ++i) ms[i] = 0.0f;
    return QS_OK;
}

qs_status qs_project(qs_plan p, const float* x, int64_t N, float* u_out, int64_t ldu, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_project: NULL plan");
    if (N < 0 || N > (p->desc.max_n > p->desc.max_m ? p->desc.max_n : p->desc.max_m) || ldu < N)
        return fail(QS_ERR_ARG, "qs_project: bad size");
    if (N > 0 && (!x || !u_out)) return fail(QS_ERR_ARG, "qs_project: NULL data pointer");
    if (N == 0) return QS_OK;
    if (!p->d_U) return fail(QS_ERR_UNSUPPORTED, "qs_project: the fused form keeps no projection workspace");
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = project(p, x, N, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_project: projection");
    e = cudaMemcpy2DAsync(u_out, (size_t)ldu * sizeof(float), p->d_U, (size_t)p->ldU * sizeof(float),
                          (size_t)N * sizeof(float), (size_t)p->desc.P, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_project: copy");
}

namespace {
qs_status sorted_call(qs_plan p, const float* x, int64_t N, const float* w, const float* y, int64_t M, float* s,
                      const float* v, float* gy, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_sum_sorted: NULL plan");
    if (p->desc.kernel != QS_NEGDIST)
        return fail(QS_ERR_UNSUPPORTED, "qs_sum_sorted: sorting slicing is for the negative distance kernel");
    if (p->desc.d > QS_FUSED_MAX_D)
        return fail(QS_ERR_UNSUPPORTED, "qs_sum_sorted: d must be <= %d", QS_FUSED_MAX_D);
    if (N < 0 || M < 0 || N > p->desc.max_n || M > p->desc.max_m)
        return fail(QS_ERR_ARG, "qs_sum_sorted: sizes outside the plan's limits");
    if ((N > 0 && !x) || (M > 0 && (!y || (!s && !gy)))) return fail(QS_ERR_ARG, "qs_sum_sorted: NULL data pointer");
    if (p->desc.max_n + p->desc.max_m > (int64_t)1 << 31)
        return fail(QS_ERR_UNSUPPORTED, "qs_sum_sorted: max_n + max_m beyond 2^31");
    if (M == 0) return QS_OK;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->d_sortws) {
        const size_t bytes = qs_sort_workspace_bytes(p->desc.P, p->desc.max_n, p->desc.max_m);
        if (cudaMalloc(&p->d_sortws, bytes) != cudaSuccess) {
            p->d_sortws = nullptr;
            return fail(QS_ERR_OOM, "qs_sum_sorted: workspace of %zu bytes", bytes);
        }
    }
    const int d = p->desc.d;
    const double cd = exp(0.5 * log(kPi) + lgamma(0.5 * (d + 1)) - lgamma(0.5 * d));
    const double amp = -cd / ((double)p->G * p->tau);  // f(t) = -c_d |t|, keys in grid units G tau <., xi>
    const float scale = (float)(-cd / p->desc.P);
    cudaError_t e = qs_launch_sum_sorted(x, N, w, y, M, p->d_dirs_s, p->d_dirs, d, p->desc.P, amp, p->d_sortws,
                                         p->desc.max_n, p->desc.max_m, s, v, scale, gy, p->d_flag, st);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_sum_sorted");
}
}  // namespace

qs_status qs_sum_sorted(qs_plan p, const float* x, int64_t N, const float* w, const float* y, int64_t M, float* s,
                        void* stream)
{
    if (M > 0 && !s) return fail(QS_ERR_ARG, "qs_sum_sorted: NULL output");
    return sorted_call(p, x, N, w, y, M, s, nullptr, nullptr, stream);
}

qs_status qs_grad_sorted(qs_plan p, const float* x, int64_t N, const float* w, const float* y, int64_t M,
                         const float* v, float* gy, void* stream)
{
    if (M > 0 && !gy) return fail(QS_ERR_ARG, "qs_grad_sorted: NULL output");
    return sorted_call(p, x, N, w, y, M, nullptr, v, gy, stream);
}

qs_status qs_grad(qs_plan p, const float* x, int64_t N, const float* w, const float* y, int64_t M, const float* v,
                  float* gx, float* gw, float* gy, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_grad: NULL plan");
    if (N < 0 || M < 0 || N > p->desc.max_n || M > p->desc.max_m)
        return fail(QS_ERR_ARG, "qs_grad: sizes outside the plan's limits");
    if ((N > 0 && !x) || (M > 0 && !y)) return fail(QS_ERR_ARG, "qs_grad: NULL point array");
    if (!gx && !gw && !gy) return QS_OK;
    if (!p->d_H2)
        return fail(QS_ERR_UNSUPPORTED, "qs_grad: the fused projection form needs d <= %d for gradients (the plan "
                    "has d = %d); use an unfused form (FP32, BF16X3, TF32)", QS_GRAD_MAX_D, p->desc.d);
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int d = p->desc.d;
    const float scale = (float)(p->tau / (double)p->desc.P);
    // unfused plans project sources and targets with their GEMM into U first
    const bool fused = p->proj == QS_PROJ_FP32_FUSED;
    // unfused forms: the derivative values q_{m,p} are written over the
    // projections in U and back-projected onto the directions by a GEMM (faster
    // than d compensated sums per target-slice at any d: 2.07 against 2.36 ms per
    // MMD-flow step at d = 16 with the 64-wide tile); the fused form has no U and
    // keeps the per-component sums (d <= QS_GRAD_MAX_D)
    const bool gemm_bp = !fused;
    cudaError_t e = cudaSuccess;
    // dL/dy_m = (tau/P) v_m sum_p xi_p sum_n w_n g'(b_{m,p} - a_{n,p}): sources x, targets y
    if (gy && M > 0) {
        if (N == 0) {
            e = cudaMemsetAsync(gy, 0, (size_t)M * d * sizeof(float), st);
        } else {
            qs_launch L = make_launch(p, N, M, 256);
            e = qs_launch_weight_scale(L, w, st);
            if (e == cudaSuccess && !fused) e = project(p, x, N, st);
            if (e == cudaSuccess) e = qs_launch_spread_grad(L, p->W, x, w, 1, fused, p->d_Dd, p->d_H2, st);
            if (e == cudaSuccess && !fused) e = project(p, y, M, st);
            if (gemm_bp) {
                if (e == cudaSuccess) e = qs_launch_interp_deriv(L, p->W, p->d_H2, st);
                if (e == cudaSuccess)
                    e = qs_launch_backproj(p->d_U, p->ldU, M, p->desc.P, p->d_dirs, d, scale, v, gy, st);
            } else {
                if (e == cudaSuccess)
                    e = qs_launch_interp_grad(L, p->W, y, p->d_H2, p->d_dirs, p->d_gpart, fused, st);
                if (e == cudaSuccess) e = qs_launch_reduce_grad(p->d_gpart, L.S, M, d, scale, v, gy, st);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "qs_grad: gradient in y");
    }
    // dL/dx_n = (tau/P) w_n sum_p xi_p sum_m v_m g'(a_{n,p} - b_{m,p}) and
    // dL/dw_n = (1/P) sum_p sum_m v_m g(a_{n,p} - b_{m,p}): sources y (weights v), targets x
    if ((gx || gw) && N > 0) {
        if (M == 0) {
            if (gx) e = cudaMemsetAsync(gx, 0, (size_t)N * d * sizeof(float), st);
            if (e == cudaSuccess && gw) e = cudaMemsetAsync(gw, 0, (size_t)N * sizeof(float), st);
        } else {
            // gw uses the (fused) interpolation kernel, gx the gradient kernel: each
            // gets the slice-group count matching its CTA shape
            qs_launch L = make_launch(p, M, N, 256);
            qs_launch Lw = make_launch(p, M, N, 256 * qs_interp_tpt(fused, p->desc.d, p->G));
            e = qs_launch_weight_scale(L, v, st);
            if (e == cudaSuccess && !fused) e = project(p, y, M, st);
            if (e == cudaSuccess) {
                if (gx)
                    e = qs_launch_spread_grad(L, p->W, y, v, gw ? 2 : 1, fused, p->d_Dd, p->d_H2, st);
                else
                    e = qs_launch_spread(L, p->W, y, v, fused, st);
            }
            if (e == cudaSuccess && !fused) e = project(p, x, N, st);
            if (gemm_bp) {
                // the plain interpolation reads the projections before the
                // derivative values overwrite them
                if (e == cudaSuccess && gw) e = qs_launch_interp(Lw, p->W, x, fused, st);
                if (e == cudaSuccess && gw) e = qs_launch_reduce(Lw, gw, st);
                if (e == cudaSuccess && gx) e = qs_launch_interp_deriv(L, p->W, p->d_H2, st);
                if (e == cudaSuccess && gx)
                    e = qs_launch_backproj(p->d_U, p->ldU, N, p->desc.P, p->d_dirs, d, scale, w, gx, st);
            } else {
                if (e == cudaSuccess && gx)
                    e = qs_launch_interp_grad(L, p->W, x, p->d_H2, p->d_dirs, p->d_gpart, fused, st);
                if (e == cudaSuccess && gx) e = qs_launch_reduce_grad(p->d_gpart, L.S, N, d, scale, w, gx, st);
                if (e == cudaSuccess && gw) e = qs_launch_interp(Lw, p->W, x, fused, st);
                if (e == cudaSuccess && gw) e = qs_launch_reduce(Lw, gw, st);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "qs_grad: gradients in x / w");
    }
    return QS_OK;
}

qs_status qs_plan_set_variant(qs_plan p, int v)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_set_variant: NULL plan");
    if (v < 0 || v >= QS_SPREAD_NVARIANTS) return fail(QS_ERR_ARG, "qs_plan_set_variant: variant %d out of range", v);
    if (!qs_spread_variant_ok(p->G, p->W, v))
        return fail(QS_ERR_ARG, "qs_plan_set_variant: variant %d is not in this plan's family (%s spread for G = %d, W = %d)",
                    v, qs_spread_moments(p->G, p->W) ? "moment" : "tap", p->G, p->W);
    p->spread_variant = v;
    return QS_OK;
}

qs_status qs_plan_set_gemm(qs_plan p, int pair)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_set_gemm: NULL plan");
    if (pair != 0 && pair != 1) return fail(QS_ERR_ARG, "qs_plan_set_gemm: pair must be 0 or 1");
    if (pair) {
        if (p->proj != QS_PROJ_BF16X3 && p->proj != QS_PROJ_TF32)
            return fail(QS_ERR_UNSUPPORTED, "qs_plan_set_gemm: the SM-pair GEMM needs a tensor-core projection");
        DeviceGuard g(p->device);
        if (!qs_tc_pair_available(p->proj == QS_PROJ_BF16X3 ? 0 : 1))
            return fail(QS_ERR_UNSUPPORTED, "qs_plan_set_gemm: two-CTA clusters of the GEMM cannot be resident");
    }
    p->gemm_pair = pair != 0;
    return QS_OK;
}

qs_status qs_plan_gemm(qs_plan p, int* pair, int* ctas)
{
    if (!p || !pair) return fail(QS_ERR_ARG, "qs_plan_gemm: NULL argument");
    *pair = p->gemm_pair ? 1 : 0;
    if (ctas) {
        DeviceGuard g(p->device);
        *ctas = p->gemm_pair ? qs_tc_pair_ctas(p->proj == QS_PROJ_BF16X3 ? 0 : 1) : p->sm_count;
    }
    return QS_OK;
}

qs_status qs_plan_variants(qs_plan p, unsigned int* available, int* current)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_variants: NULL plan");
    unsigned int mask = 0;
    for (int v = 0; v < QS_SPREAD_NVARIANTS; ++v)
        if (qs_spread_variant_ok(p->G, p->W, v)) mask |= 1u << v;
    if (available) *available = mask;
    if (current) *current = p->spread_variant;
    return QS_OK;
}

qs_status qs_plan_autotune(qs_plan p, const float* x, int64_t N, const float* w, int* chosen, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_autotune: NULL plan");
    if (N <= 0 || N > (p->desc.max_n > p->desc.max_m ? p->desc.max_n : p->desc.max_m) || !x)
        return fail(QS_ERR_ARG, "qs_plan_autotune: need 0 < N <= max(max_n, max_m) sources");
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool fused = p->proj == QS_PROJ_FP32_FUSED;
    qs_launch L = make_launch(p, N, 1, 256);
    cudaError_t e = cudaSuccess;
    if (!fused) e = project(p, x, N, st);
    if (e == cudaSuccess) e = qs_launch_weight_scale(L, w, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_plan_autotune: setup");
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(QS_ERR_CUDA, "qs_plan_autotune: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(QS_ERR_CUDA, "qs_plan_autotune: event");
    }
    int best = qs_spread_default(p->G, p->W);
    float best_ms = 3.4e38f;
    for (int v = 0; v < QS_SPREAD_NVARIANTS && e == cudaSuccess; ++v) {
        if (!qs_spread_variant_ok(p->G, p->W, v)) continue;
        L.spread_variant = v;
        e = qs_launch_spread(L, p->W, x, w, fused, st);  // warm-up
        float vbest = 3.4e38f;
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = qs_launch_spread(L, p->W, x, w, fused, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (ms < vbest) vbest = ms;
        }
        if (vbest < best_ms) {
            best_ms = vbest;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "qs_plan_autotune: timing");
    p->spread_variant = best;
    qs_tune_store(p, best, -1);
    if (chosen) *chosen = best;
    return QS_OK;
}

qs_status qs_plan_autotune_gemm(qs_plan p, const float* x, int64_t N, int* chosen, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_plan_autotune_gemm: NULL plan");
    if (N <= 0 || N > (p->desc.max_n > p->desc.max_m ? p->desc.max_n : p->desc.max_m) || !x)
        return fail(QS_ERR_ARG, "qs_plan_autotune_gemm: need 0 < N <= max(max_n, max_m) points");
    if (p->proj != QS_PROJ_BF16X3 && p->proj != QS_PROJ_TF32)
        return fail(QS_ERR_UNSUPPORTED, "qs_plan_autotune_gemm: the plan has no tensor-core projection");
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool pair_ok = qs_tc_pair_available(p->proj == QS_PROJ_BF16X3 ? 0 : 1);
    const bool keep = p->gemm_pair;
    cudaError_t e = project_prep(p, x, N, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_plan_autotune_gemm: operand split");
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(QS_ERR_CUDA, "qs_plan_autotune_gemm: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(QS_ERR_CUDA, "qs_plan_autotune_gemm: event");
    }
    int best = keep ? 1 : 0;
    float best_ms = 3.4e38f;
    for (int pair = 0; pair <= (pair_ok ? 1 : 0) && e == cudaSuccess; ++pair) {
        p->gemm_pair = pair == 1;
        e = project_gemm(p, x, N, st);  // warm-up
        float vbest = 3.4e38f;
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = project_gemm(p, x, N, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (ms < vbest) vbest = ms;
        }
        if (vbest < best_ms) {
            best_ms = vbest;
            best = pair;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        p->gemm_pair = keep;
        return cuda_fail(e, "qs_plan_autotune_gemm: timing");
    }
    p->gemm_pair = best == 1;
    qs_tune_store(p, -1, best);
    if (chosen) *chosen = best;
    return QS_OK;
}

qs_status qs_check(qs_plan p, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_check: NULL plan");
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int flag = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_check: stream");
    e = cudaMemcpy(&flag, p->d_flag, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qs_check: read flag");
    e = cudaMemset(p->d_flag, 0, sizeof(flag));
    if (e != cudaSuccess) return cuda_fail(e, "qs_check: clear flag");
    if (flag & QS_FLAG_TIMEOUT) return fail(QS_ERR_TIMEOUT, "device wait timed out");
    if (flag & QS_FLAG_NONFINITE) return fail(QS_ERR_NONFINITE, "NaN or Inf in the inputs");
    if (flag & QS_FLAG_RANGE) return fail(QS_ERR_RANGE, "a projection exceeded the half period; increase radius");
    return QS_OK;
}

qs_status qs_sum_host(qs_plan p, const float* xh, int64_t N, const float* wh, const float* yh, int64_t M,
                      float* sh, void* stream)
{
    if (!p) return fail(QS_ERR_ARG, "qs_sum_host: NULL plan");
    if (N < 0 || M < 0 || N > p->desc.max_n || M > p->desc.max_m)
        return fail(QS_ERR_ARG, "qs_sum_host: sizes outside the plan's limits");
    if ((N > 0 && !xh) || (M > 0 && (!yh || !sh))) return fail(QS_ERR_ARG, "qs_sum_host: NULL data pointer");
    if (M == 0) return QS_OK;
    DeviceGuard g(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int d = p->desc.d;
    cudaError_t e = cudaSuccess;
    if (N == 0 || p->timing) {
        // serial form: the stage timers of qs_sum stay meaningful
        if (N > 0) e = cudaMemcpyAsync(p->d_x, xh, (size_t)N * d * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && N > 0 && wh)
            e = cudaMemcpyAsync(p->d_w, wh, (size_t)N * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_y, yh, (size_t)M * d * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: copy in");
        qs_status rs = qs_sum(p, p->d_x, N, wh ? p->d_w : nullptr, p->d_y, M, p->d_s, stream);
        if (rs != QS_OK) return rs;
    } else {
        // pipelined form: x, then y, arrive in row chunks on the plan's copy
        // stream; each chunk is projected on `stream` as soon as it has
        // landed, and each y chunk also interpolated, so the transfer of x
        // overlaps its GEMM and the transfer of y the spread and the GEMM
        // and interpolation of the chunks before it.  x comes in up to
        // QS_HOST_CHUNKS chunks, y in QS_HOST_Y_CHUNKS: the slice groups are
        // fixed by M, so an interpolation launch over a smaller chunk has
        // fewer CTAs and wastes part of its waves.  y chunks are
        // whole interpolation CTAs (256 x targets per thread), so every CTA
        // sees the targets it sees in qs_sum and the results are the same bits
        if (!p->copy_st) {
            e = cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking);
            for (int i = 0; e == cudaSuccess && i < 1 + 2 * QS_HOST_CHUNKS; ++i)
                e = cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: copy stream");
        }
        cudaStream_t cs = p->copy_st;
        cudaEvent_t* ex = p->hev + 1;
        cudaEvent_t* ey = p->hev + 1 + QS_HOST_CHUNKS;
        const bool fused = p->proj == QS_PROJ_FP32_FUSED;
        const int64_t cx = host_chunk_rows(N),
                      cy = host_chunk_rows(M, 256 * qs_interp_tpt(fused, d, p->G), QS_HOST_Y_CHUNKS);
        const int nx = (int)((N + cx - 1) / cx), ny = (int)((M + cy - 1) / cy);
        // the copies wait for the work already queued on `stream` (it may read the staging buffers)
        e = cudaEventRecord(p->hev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, p->hev[0], 0);
        if (e == cudaSuccess && wh) e = cudaMemcpyAsync(p->d_w, wh, (size_t)N * sizeof(float), cudaMemcpyHostToDevice, cs);
        for (int i = 0; e == cudaSuccess && i < nx; ++i) {
            const int64_t r0 = i * cx, r = (N - r0 < cx ? N - r0 : cx);
            e = cudaMemcpyAsync(p->d_x + r0 * d, xh + r0 * d, (size_t)r * d * sizeof(float), cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ex[i], cs);
        }
        for (int i = 0; e == cudaSuccess && i < ny; ++i) {
            const int64_t r0 = i * cy, r = (M - r0 < cy ? M - r0 : cy);
            e = cudaMemcpyAsync(p->d_y + r0 * d, yh + r0 * d, (size_t)r * d * sizeof(float), cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ey[i], cs);
        }
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: copy in");
        qs_launch L = make_launch(p, N, M, 256 * qs_interp_tpt(fused, d, p->G));
        if (fused) e = cudaStreamWaitEvent(st, ex[nx - 1], 0);
        for (int i = 0; !fused && e == cudaSuccess && i < nx; ++i) {
            const int64_t r0 = i * cx, r = (N - r0 < cx ? N - r0 : cx);
            e = cudaStreamWaitEvent(st, ex[i], 0);
            if (e == cudaSuccess) e = project_rows(p, p->d_x, r0, r, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: projection of x");
        e = qs_launch_weight_scale(L, wh ? p->d_w : nullptr, st);
        if (e == cudaSuccess) e = qs_launch_spread(L, p->W, p->d_x, wh ? p->d_w : nullptr, fused, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: spread");
        for (int i = 0; e == cudaSuccess && i < ny; ++i) {
            const int64_t r0 = i * cy, r = (M - r0 < cy ? M - r0 : cy);
            e = cudaStreamWaitEvent(st, ey[i], 0);
            if (e == cudaSuccess && !fused) e = project_rows(p, p->d_y, r0, r, st);
            if (e == cudaSuccess) {
                qs_launch Li = L;
                Li.m_base = r0;
                Li.m_end = r0 + r;
                e = qs_launch_interp(Li, p->W, p->d_y, fused, st);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: projection and interpolation of y");
        e = qs_launch_reduce(L, p->d_s, st);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: reduction");
    }
    e = cudaMemcpyAsync(sh, p->d_s, (size_t)M * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sum_host: copy out");
    return qs_check(p, stream);
}

}  // extern "C"
