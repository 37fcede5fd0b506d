// qs_sum_noalloc: the fast kernel sum for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or unwanted --
// a host framework whose caching allocator owns all device memory and
// forbids outside allocations, a real-time or inference loop that must not
// pay for (or synchronise on) an allocation, or a plugin that is handed
// input and output buffers and nothing else.  Such a caller cannot create a
// plan, because plan creation allocates its workspace.
//
// What it does: the same sum as qs_sum with the fused FP32 projection
// (d <= 64), but every intermediate -- the filter table, the twiddles, the
// scaled directions, the per-slice filtered grids, the slice partial sums,
// the weight scale and the error flag -- lives in one file-scope device
// array of QS_NOALLOC_SCRATCH_BYTES (16 MiB).  Every GPU that loads the
// library holds that array until the process exits.  No call allocates.
//
// Sharing: all calls on a device use the same array and it keeps the last
// call's contents; each call rewrites everything it reads (the error flag is
// cleared at the start).  Calls whose GPU work overlaps -- concurrent streams
// or host threads on the same device -- race on the array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "qs_internal.cuh"

#define QS_NOALLOC_SCRATCH_BYTES (16u << 20)
#define QS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[QS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

std::mutex g_setup_mutex;
void* g_scratch_ptr[QS_NOALLOC_MAX_DEVICES] = {nullptr};

qs_status nfail(qs_status st, const char* fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    qs_set_error_message(msg);
    return st;
}

// Device address of the scratch array on the current device.  The array's
// name in host code is only a stand-in; the address is looked up once per
// device (first call on that device) and cached.
cudaError_t scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= QS_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

// ---- heap-free host tables (same arithmetic as plan creation) -------------
double es(double v, int m, double beta)
{
    const double z = v / m;
    if (fabs(z) >= 1.0) return 0.0;
    return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

void gl24(double* x, double* w)
{
    const int n = 24;
    for (int i = 0; i < n; ++i) {
        double t = cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 1; j < n; ++j) {
                const double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

void fit(int W, double beta, qs_window& win)
{
    const int m = W / 2;
    const int n = qs_tap_degree(W) + 1;
    double tm[QS_MAX_W + 2][QS_MAX_W + 2];
    memset(&win, 0, sizeof(win));
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) tm[k][i] = 0.0;
    tm[0][0] = 1.0;
    tm[1][1] = 2.0;
    for (int k = 2; k < n; ++k)
        for (int i = 0; i < n; ++i) {
            double v = -tm[k - 2][i];
            if (i > 0) v += 4.0 * tm[k - 1][i - 1];
            tm[k][i] = v;
        }
    for (int j = 0; j < m; ++j) {
        double cheb[QS_MAX_W + 2], fval[QS_MAX_W + 2], mono[QS_MAX_W + 2];
        for (int i = 0; i < n; ++i) fval[i] = es(0.5 * cos(kPi * (i + 0.5) / n) + m - 0.5 - j, m, beta);
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += fval[i] * cos(k * kPi * (i + 0.5) / n);
            cheb[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
        }
        for (int i = 0; i < n; ++i) mono[i] = 0.0;
        for (int k = 0; k < n; ++k)
            for (int i = 0; i < n; ++i) mono[i] += cheb[k] * tm[k][i];
        for (int i = 0; i < n; ++i) {
            if (i % 2 == 0) win.e[j][i / 2] = (float)mono[i];
            else win.o[j][i / 2] = (float)mono[i];
        }
    }
}

double tap(const qs_window& win, int W, int j, double s)
{
    const int m = W / 2, T = qs_tap_terms(W);
    const int jj = j < m ? j : W - 1 - j;
    const double ss = j < m ? s : -s;
    double e = 0.0, o = 0.0;
    for (int i = T - 1; i >= 0; --i) {
        e = e * ss * ss + (double)win.e[jj][i];
        o = o * ss * ss + (double)win.o[jj][i];
    }
    return e + ss * o;
}

// Per-call host staging of the small tables (no heap): window transform
// (K + 1 doubles) and twiddles (G/2 float2).  Serialised by g_setup_mutex.
double g_psihat[QS_MAX_G / 4 + 1];
float2 g_tw[QS_MAX_G / 2];

__global__ void scale_dirs_kernel(const float* __restrict__ dirs, int64_t n, double scale, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(scale * (double)dirs[i]);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" qs_status qs_sum_noalloc(const qs_plan_desc* desc, const float* dirs_dev, const float* x, int64_t N,
                                    const float* w, const float* y, int64_t M, float* s, void* stream)
{
    if (!desc || !dirs_dev) return nfail(QS_ERR_ARG, "qs_sum_noalloc: NULL desc or directions");
    const qs_plan_desc& D = *desc;
    if (D.d < 1 || D.d > QS_FUSED_MAX_D || D.P < 1)
        return nfail(QS_ERR_ARG, "qs_sum_noalloc: need 1 <= d <= %d and P >= 1", QS_FUSED_MAX_D);
    if (D.kernel < QS_GAUSS || D.kernel > QS_TPS)
        return nfail(QS_ERR_ARG, "qs_sum_noalloc: unknown kernel");
    if (D.kernel == QS_RIESZ || D.kernel == QS_TPS)
        return nfail(QS_ERR_UNSUPPORTED,
                     "qs_sum_noalloc: the Riesz and thin plate spline coefficients need a plan (host quadrature)");
    if (D.kernel != QS_NEGDIST && !(D.kparam > 0.0 && isfinite(D.kparam)))
        return nfail(QS_ERR_ARG, "qs_sum_noalloc: kernel parameter must be positive");
    if (D.kernel == QS_MATERN && !(D.kparam2 > 0.0 && D.kparam2 < 1e6))
        return nfail(QS_ERR_ARG, "qs_sum_noalloc: Matern nu (kparam2) must be positive");
    if (!(D.radius > 0.0 && isfinite(D.radius))) return nfail(QS_ERR_ARG, "qs_sum_noalloc: radius must be > 0");
    if (D.n_ft < 16 || D.n_ft > QS_MAX_G / 2 || (D.n_ft & (D.n_ft - 1)))
        return nfail(QS_ERR_UNSUPPORTED, "qs_sum_noalloc: n_ft must be a power of two in [16, %d]", QS_MAX_G / 2);
    const int W = D.window == 0 ? 8 : D.window;
    if (W != 6 && W != 8 && W != 10 && W != 12) return nfail(QS_ERR_UNSUPPORTED, "qs_sum_noalloc: bad window");
    if (D.oversampling != 0.0 && D.oversampling != 2.0)
        return nfail(QS_ERR_UNSUPPORTED, "qs_sum_noalloc: only oversampling 2 is supported");
    if (D.proj != QS_PROJ_AUTO && D.proj != QS_PROJ_FP32_FUSED)
        return nfail(QS_ERR_UNSUPPORTED, "qs_sum_noalloc: only the fused FP32 projection is available");
    if (N < 0 || M < 0) return nfail(QS_ERR_ARG, "qs_sum_noalloc: negative size");
    if ((N > 0 && !x) || (M > 0 && (!y || !s))) return nfail(QS_ERR_ARG, "qs_sum_noalloc: NULL data pointer");
    if (M == 0) return QS_OK;

    const int G = 2 * D.n_ft, K = D.n_ft / 2, d = D.d, P = D.P;
    // slice groups as in qs_sum, reduced only if the partial sums do not fit
    const int S_max = P < 64 ? P : 64;
    const int64_t blocks_m = (M + 255) / 256;
    int64_t S = (1024 + blocks_m - 1) / blocks_m;
    if (S > S_max) S = S_max;
    if (S < 1) S = 1;
    const size_t o_flag = 0, o_wscale = 256, o_psihat = 512;
    const size_t o_c = o_psihat + align256((size_t)(K + 1) * 8);
    const size_t o_D = o_c + align256((size_t)D.n_ft * 8);
    const size_t o_tw = o_D + align256((size_t)(G / 2 + 1) * 4);
    const size_t o_xi = o_tw + align256((size_t)(G / 2) * 8);
    const size_t o_H = o_xi + align256((size_t)P * d * 4);
    const size_t o_part = o_H + align256((size_t)P * G * 4);
    const size_t avail = o_part < QS_NOALLOC_SCRATCH_BYTES ? QS_NOALLOC_SCRATCH_BYTES - o_part : 0;
    while (S > 1 && (size_t)(2 * S) * (size_t)M * 4 > avail) --S;
    const size_t need = o_part + (size_t)(2 * S) * (size_t)M * 4;
    if (need > QS_NOALLOC_SCRATCH_BYTES)
        return nfail(QS_ERR_UNSUPPORTED,
                     "qs_sum_noalloc: needs %zu bytes of scratch (P=%d, G=%d, M=%lld) but the static scratch "
                     "holds %u bytes; use a plan (qs_plan_create / qs_sum) for this size",
                     need, P, G, (long long)M, (unsigned)QS_NOALLOC_SCRATCH_BYTES);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return nfail(QS_ERR_CUDA, "qs_sum_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;

    double tau;
    switch (D.kernel) {
        case QS_GAUSS: tau = fmin(0.3 / D.radius, 1.0 / (2.0 * 5.0 * D.kparam)); break;
        case QS_LAPLACE: tau = fmin(0.1 / D.radius, 1.0 / (2.0 * 5.0 / D.kparam)); break;
        case QS_MATERN: tau = fmin(0.2 / D.radius, 1.0 / (2.0 * 5.0 * D.kparam)); break;
        default: tau = 1.0 / (2.0 * D.radius); break;
    }
    qs_launch L;
    memset(&L, 0, sizeof(L));
    L.d = d;
    L.P = P;
    L.G = G;
    L.n_ft = D.n_ft;
    L.N = N;
    L.M = M;
    L.m_base = 0;
    L.m_end = M;
    L.ldU = 0;
    L.half_G = 0.5f * (float)G;
    L.xi_s = reinterpret_cast<const float*>(base + o_xi);
    L.D = reinterpret_cast<const float*>(base + o_D);
    L.tw = reinterpret_cast<const float2*>(base + o_tw);
    L.H = reinterpret_cast<float*>(base + o_H);
    L.U = nullptr;
    L.part = reinterpret_cast<float*>(base + o_part);
    L.S = (int)S;
    L.spread_variant = qs_spread_default(G, W);
    L.flag = reinterpret_cast<unsigned int*>(base + o_flag);
    L.wscale = reinterpret_cast<float*>(base + o_wscale);

    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        fit(W, 2.30 * W, L.win);
        double gx[24], gw[24];
        gl24(gx, gw);
        for (int k = 0; k <= K; ++k) {
            const double nu = (double)k / G;
            double acc = 0.0;
            for (int j = 0; j < W; ++j) {
                const double c = W / 2 - 0.5 - j;
                for (int q = 0; q < 24; ++q) {
                    const double sq = 0.5 * gx[q];
                    acc += 0.5 * gw[q] * tap(L.win, W, j, sq) * cos(2.0 * kPi * nu * (sq + c));
                }
            }
            g_psihat[k] = acc;
        }
        for (int t = 0; t < G / 2; ++t) {
            const double ang = 2.0 * kPi * (double)t / (double)G;
            g_tw[t] = make_float2((float)cos(ang), (float)(-sin(ang)));
        }
        // pageable source: each copy has been staged when the call returns, so
        // the host tables may be rewritten by the next call
        e = cudaMemcpyAsync(base + o_psihat, g_psihat, (size_t)(K + 1) * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_tw, g_tw, (size_t)(G / 2) * 8, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: table upload: %s", cudaGetErrorString(e));
    e = cudaMemsetAsync(base + o_flag, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: clear flag: %s", cudaGetErrorString(e));
    const int64_t nd = (int64_t)P * d;
    scale_dirs_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(dirs_dev, nd, (double)G * tau,
                                                                     reinterpret_cast<float*>(base + o_xi));
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = qs_launch_coeffs((int)D.kernel, D.kparam, D.kparam2, d, tau, D.n_ft, G,
                             reinterpret_cast<const double*>(base + o_psihat), nullptr,
                             reinterpret_cast<double*>(base + o_c), reinterpret_cast<float*>(base + o_D), st);
    if (e == cudaSuccess) {
        if (N == 0) {
            e = cudaMemsetAsync(s, 0, (size_t)M * sizeof(float), st);
        } else {
            e = qs_launch_weight_scale(L, w, st);
            if (e == cudaSuccess) e = qs_launch_spread(L, W, x, w, true, st);
            if (e == cudaSuccess) e = qs_launch_interp(L, W, y, true, st);
            if (e == cudaSuccess) e = qs_launch_reduce(L, s, st);
        }
    }
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: launch: %s", cudaGetErrorString(e));
    unsigned int flag = 0;
    e = cudaMemcpyAsync(&flag, base + o_flag, sizeof(flag), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: %s", cudaGetErrorString(e));
    if (flag & QS_FLAG_TIMEOUT) return nfail(QS_ERR_TIMEOUT, "qs_sum_noalloc: device wait timed out");
    if (flag & QS_FLAG_NONFINITE) return nfail(QS_ERR_NONFINITE, "qs_sum_noalloc: NaN or Inf in the inputs");
    if (flag & QS_FLAG_RANGE) return nfail(QS_ERR_RANGE, "qs_sum_noalloc: a projection exceeded the half period");
    qs_set_error_message("");
    return QS_OK;
}
