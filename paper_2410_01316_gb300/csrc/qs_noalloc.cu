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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "qs_internal.cuh"

#define QS_NOALLOC_SCRATCH_BYTES (16u << 20)
#define QS_NOALLOC_MAX_DEVICES 64
#define QS_NOALLOC_TABLE_CACHE 4

static __device__ __align__(256) unsigned char g_noalloc_scratch[QS_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;

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

// ---- device address of the scratch array -----------------------------------
// In host code the array's name is only a stand-in, not a device address.
// The address is looked up with cudaGetSymbolAddress once per device, with
// that device current, and cached together with the identity of the device's
// context: after a cudaDeviceReset the module is loaded again (possibly at
// another address), the context identity changes and the lookup is repeated.
struct ScratchEntry {
    void* ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool has_id = false;
};
ScratchEntry g_scratch[QS_NOALLOC_MAX_DEVICES];

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
bool g_ctx_fns_looked_up = false;

// Identity of the calling thread's current context; false if it cannot be read.
bool current_context_id(unsigned long long* id)
{
    if (!g_ctx_fns_looked_up) {
        g_ctx_fns_looked_up = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    }
    if (!g_ctx_current || !g_ctx_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

// Caller holds g_setup_mutex; the device `dev` is current (the runtime has
// made its primary context current by the time this runs).
cudaError_t scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= QS_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    ScratchEntry& e = g_scratch[dev];
    unsigned long long id = 0;
    const bool has_id = current_context_id(&id);
    if (!e.ptr || !has_id || !e.has_id || e.ctx_id != id) {
        void* ptr = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (err != cudaSuccess) {
            e.ptr = nullptr;
            return err;
        }
        e.ptr = ptr;
        e.has_id = has_id;
        e.ctx_id = id;
    }
    *out = static_cast<unsigned char*>(e.ptr);
    return cudaSuccess;
}

// ---- host tables, cached per (W, G) ------------------------------------------
// The tap polynomials, the window transform (K + 1 = G/4 + 1 values) and the
// twiddles depend only on the window (width W, kind) and the grid size G.  They are
// computed by the same host code as at plan creation (qs_tables.cu), so both
// entry points use bitwise identical tables, and kept in a few static slots
// (no heap) so repeated calls with the same sizes do not recompute them.
struct TableEntry {
    int W = 0, G = 0, kind = -1;
    qs_window win;
    double psihat[QS_MAX_G / 4 + 1];
    float2 tw[QS_MAX_G / 2];
};
TableEntry g_tables[QS_NOALLOC_TABLE_CACHE];
int g_tables_next = 0;

// Caller holds g_setup_mutex.
const TableEntry& tables_for(int W, int kind, int G)
{
    for (auto& t : g_tables)
        if (t.W == W && t.G == G && t.kind == kind) return t;
    TableEntry& t = g_tables[g_tables_next];
    g_tables_next = (g_tables_next + 1) % QS_NOALLOC_TABLE_CACHE;
    qs_fit_window(W, kind, &t.win);
    qs_window_transform(&t.win, W, G / 4, G, t.psihat);
    qs_twiddles(G, t.tw);
    t.W = W;
    t.G = G;
    t.kind = kind;
    return t;
}

// Directions scaled by G tau, in the same FP64 product and FP32 rounding as at
// plan creation; a non-finite direction entry sets the data-error flag.
__global__ void scale_dirs_kernel(const float* __restrict__ dirs, int64_t n, double scale, float* __restrict__ out,
                                  unsigned int* flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float v = dirs[i];
        if (!isfinite(v)) {
            atomicOr(flag, QS_FLAG_NONFINITE);
            out[i] = 0.0f;
        } else {
            out[i] = (float)(scale * (double)v);
        }
    }
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
    if (D.window_kind != QS_WINDOW_ES && D.window_kind != QS_WINDOW_KB)
        return nfail(QS_ERR_ARG, "qs_sum_noalloc: unknown window kind");
    if (D.proj != QS_PROJ_AUTO && D.proj != QS_PROJ_FP32_FUSED)
        return nfail(QS_ERR_UNSUPPORTED, "qs_sum_noalloc: only the fused FP32 projection is available");
    if (N < 0 || M < 0) return nfail(QS_ERR_ARG, "qs_sum_noalloc: negative size");
    if ((N > 0 && !x) || (M > 0 && (!y || !s))) return nfail(QS_ERR_ARG, "qs_sum_noalloc: NULL data pointer");
    if (M == 0) return QS_OK;

    const int G = 2 * D.n_ft, K = D.n_ft / 2, d = D.d, P = D.P;
    // slice groups chosen as qs_sum chooses them for the fused form (targets
    // per interpolation CTA from qs_interp_tpt), reduced only if the partial
    // sums do not fit the scratch array
    const int S_max = P < 64 ? P : 64;
    const int64_t tpc = 256 * (int64_t)qs_interp_tpt(true, d, G);
    const int64_t blocks_m = (M + tpc - 1) / tpc;
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
    cudaStream_t st = (cudaStream_t)stream;
    const double tau = qs_tau_rule(D.kernel, D.kparam, D.radius);
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
    L.U = nullptr;
    L.S = (int)S;
    L.spread_variant = qs_spread_default(G, W);

    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        e = scratch_address(dev, &base);
        if (e != cudaSuccess)
            return nfail(QS_ERR_CUDA, "qs_sum_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        const TableEntry& tb = tables_for(W, D.window_kind, G);
        L.win = tb.win;
        qs_fill_atab(&tb.win, W, L.atab);  // into the launch parameters; no allocation
        // pageable source: each copy has been staged when the call returns, so
        // the cache slot may be reused by a later call
        e = cudaMemcpyAsync(base + o_psihat, tb.psihat, (size_t)(K + 1) * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_tw, tb.tw, (size_t)(G / 2) * 8, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: table upload: %s", cudaGetErrorString(e));
    L.xi_s = reinterpret_cast<const float*>(base + o_xi);
    L.D = reinterpret_cast<const float*>(base + o_D);
    L.tw = reinterpret_cast<const float2*>(base + o_tw);
    L.H = reinterpret_cast<float*>(base + o_H);
    L.part = reinterpret_cast<float*>(base + o_part);
    L.flag = reinterpret_cast<unsigned int*>(base + o_flag);
    L.wscale = reinterpret_cast<float*>(base + o_wscale);
    e = cudaMemsetAsync(base + o_flag, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return nfail(QS_ERR_CUDA, "qs_sum_noalloc: clear flag: %s", cudaGetErrorString(e));
    const int64_t nd = (int64_t)P * d;
    scale_dirs_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(dirs_dev, nd, (double)G * tau,
                                                                     reinterpret_cast<float*>(base + o_xi), L.flag);
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
