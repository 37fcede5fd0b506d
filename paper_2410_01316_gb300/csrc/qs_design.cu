// Distance QMC designs (Sec. 2.3, eq. distance-mmd with s = d/2, and the
// symmetric form of eq. distance-sym): P unit directions xi_p minimising
//   E_sym(xi) = E((xi, -xi)) = -2 sum_{p,q} (|xi_p - xi_q| + |xi_p + xi_q|),
// the energy of the points together with their antipodes (the sliced
// integrand is even in xi, so the antipodes come for free).  As in Sec. 4.1
// the minimiser is found with Adam (on the tangential gradient, with the step
// annealed over the run); each step is followed by renormalising the rows
// onto the sphere.
//
// For unit rows |xi_p -+ xi_q|^2 = 2 -+ 2 c_pq with c = Xi Xi^T, so with
// a_pq = 1/sqrt(2 - 2c) (0 on the diagonal) and b_pq = 1/sqrt(2 + 2c):
//   dE/dxi_p = -4 [ xi_p r_p + sum_q (b_pq - a_pq) xi_q ],  r_p = sum_q (a_pq + b_pq),
// i.e. two P x P x d contractions (the Gram matrix and (B - A) Xi) done by
// the library's FP32 SIMT GEMM, plus elementwise work.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "qs_internal.cuh"

namespace {

qs_status design_fail(qs_status s, const char* msg)
{
    qs_set_error_message(msg);
    return s;
}

// Row p of the Gram matrix C (stride ldc) -> weights W = B - A in place,
// zero in the padding columns P .. ldc-1; r_p; and (ENERGY) the row's share of
// the energy, sum_q (|xi_p - xi_q| + |xi_p + xi_q|), in FP64.  One CTA per row.
// The optimiser's steps need no energy: its two FP64 square roots per pair
// would cost about as much as the step's contractions on this GPU's FP64 pipe.
template <bool ENERGY>
__global__ void __launch_bounds__(256) esym_weights_kernel(float* __restrict__ C, int P, int64_t ldc,
                                                           float* __restrict__ r, double* __restrict__ e_row)
{
    const int p = blockIdx.x;
    float* row = C + (size_t)p * ldc;
    float racc = 0.0f;
    double eacc = 0.0;
    for (int64_t q = threadIdx.x; q < ldc; q += blockDim.x) {
        if (q >= P) {
            row[q] = 0.0f;
            continue;
        }
        const float c = fminf(1.0f, fmaxf(-1.0f, row[q]));
        const float dm2 = 2.0f - 2.0f * c, dp2 = 2.0f + 2.0f * c;
        // coincident or antipodal pairs have no gradient direction: weight 0
        const float a = (q == p || dm2 <= 0.0f) ? 0.0f : rsqrtf(dm2);
        const float b = dp2 > 0.0f ? rsqrtf(dp2) : 0.0f;
        row[q] = b - a;
        racc += a + b;
        if (ENERGY) eacc += (q == p ? 0.0 : sqrt((double)dm2)) + sqrt((double)dp2);
    }
    __shared__ float rs[8];
    __shared__ double es[8];
    for (int o = 16; o > 0; o >>= 1) {
        racc += __shfl_xor_sync(0xffffffffu, racc, o);
        eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = racc;
        es[threadIdx.x >> 5] = eacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float rt = 0.0f;
        double et = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            rt += rs[i];
            et += es[i];
        }
        r[p] = rt;
        if (ENERGY) e_row[p] = et;
    }
}

// Xi (P x d) -> Xi^T (d x ldt), zero in columns P .. ldt-1.
__global__ void transpose_pad_kernel(const float* __restrict__ X, int P, int d, int64_t ldt, float* __restrict__ T)
{
    __shared__ float tile[32][33];
    const int p0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int p = p0 + i, j = j0 + threadIdx.x;
        tile[i][threadIdx.x] = (p < P && j < d) ? X[(size_t)p * d + j] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int j = j0 + i;
        const int64_t p = p0 + threadIdx.x;
        if (j < d && p < ldt) T[(size_t)j * ldt + p] = tile[threadIdx.x][i];
    }
}

// Gradient -4 (r_p xi_p + Gm_p) (Gm = (B - A) Xi, stride ldg), the Euclidean
// gradient dE/dxi_p (grad_out, may be NULL); with m, v: one Adam step on row p
// of xi along the tangential part g - <g, xi_p> xi_p (the radial part only
// changes the length, which the renormalisation discards, and would dominate
// Adam's second moment), then the renormalisation.  One CTA per row.
__device__ __forceinline__ float block_sum(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float tot = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
    return tot;
}

__global__ void __launch_bounds__(256) esym_step_kernel(float* __restrict__ xi, int d, const float* __restrict__ r,
                                                        const float* __restrict__ Gm, int64_t ldg,
                                                        float* __restrict__ grad_out, float* __restrict__ m,
                                                        float* __restrict__ v, float lr, float b1, float b2,
                                                        float b1t, float b2t, float eps)
{
    __shared__ float red[8];
    const int p = blockIdx.x;
    float* x = xi + (size_t)p * d;
    const float rp = r[p];
    float dot = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float g = -4.0f * fmaf(rp, x[j], Gm[(size_t)p * ldg + j]);
        if (grad_out) grad_out[(size_t)p * d + j] = g;
        dot = fmaf(g, x[j], dot);
    }
    if (!m) return;
    dot = block_sum(dot, red);
    float ss = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float g = -4.0f * fmaf(rp, x[j], Gm[(size_t)p * ldg + j]) - dot * x[j];
        const size_t i = (size_t)p * d + j;
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float xn = x[j] - lr * (mi / (1.0f - b1t)) / (sqrtf(vi / (1.0f - b2t)) + eps);
        x[j] = xn;
        ss = fmaf(xn, xn, ss);
    }
    const float tot = block_sum(ss, red);
    const float inv = tot > 0.0f ? rsqrtf(tot) : 1.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) x[j] *= inv;
}

// Split-K form of the second contraction Gm[p][j] = sum_q W[p][q] T[j][q]
// (W the P x ldc weights, T = Xi^T padded to ldc columns): its P x d output
// has few 128 x 128 tiles (80 at P = 5000, d = 200) for a long inner length,
// so CTA (p tile, j tile, z) sums the inner range [z kc, (z + 1) kc) into its
// own partial (parts[z], P x ldg) with the FP32 SIMT tile of the projection
// (8 x 8 outputs per thread, 8-deep slabs double-buffered in shared memory),
// and gm_reduce_kernel adds the partials in z order, so the result does not
// depend on scheduling.  kc is a multiple of the slab depth.
constexpr int SK_BM = 128, SK_BN = 128, SK_BK = 8;

__global__ void __launch_bounds__(256) gm_splitk_kernel(const float* __restrict__ Wt, int P, int64_t ldc,
                                                        const float* __restrict__ T, int d, int64_t kc,
                                                        float* __restrict__ parts, int64_t ldg)
{
    __shared__ __align__(16) float As[2][SK_BK][SK_BM];
    __shared__ __align__(16) float Bs[2][SK_BK][SK_BN];
    const int p0 = blockIdx.x * SK_BM, j0 = blockIdx.y * SK_BN;
    const int64_t k0 = (int64_t)blockIdx.z * kc;
    const int64_t k1 = k0 + kc < ldc ? k0 + kc : ldc;
    float* out = parts + (size_t)blockIdx.z * (size_t)P * ldg;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int lrow = tid >> 1, lk = (tid & 1) * 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    // slab loads: row lrow of the W tile and of the T tile, 4 consecutive inner indices from k + lk
    // as one 16-byte load (rows are 128-float aligned, k + lk is a multiple of 4, and the range end
    // k1 is a multiple of 8, so a vector lies wholly inside or outside the range)
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    auto load = [&](int64_t k, float4& ra, float4& rb) {
        const int gp = p0 + lrow, gj = j0 + lrow;
        const int64_t kk = k + lk;
        ra = (gp < P && kk < k1) ? __ldg(reinterpret_cast<const float4*>(&Wt[(size_t)gp * ldc + kk])) : zero4;
        rb = (gj < d && kk < k1) ? __ldg(reinterpret_cast<const float4*>(&T[(size_t)gj * ldc + kk])) : zero4;
    };
    auto put = [&](int buf, const float4& ra, const float4& rb) {
        As[buf][lk + 0][lrow] = ra.x;
        As[buf][lk + 1][lrow] = ra.y;
        As[buf][lk + 2][lrow] = ra.z;
        As[buf][lk + 3][lrow] = ra.w;
        Bs[buf][lk + 0][lrow] = rb.x;
        Bs[buf][lk + 1][lrow] = rb.y;
        Bs[buf][lk + 2][lrow] = rb.z;
        Bs[buf][lk + 3][lrow] = rb.w;
    };
    float4 ra, rb;
    load(k0, ra, rb);
    put(0, ra, rb);
    __syncthreads();
    const int nk = (int)((k1 - k0 + SK_BK - 1) / SK_BK);
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load(k0 + (int64_t)(kt + 1) * SK_BK, ra, rb);
#pragma unroll
        for (int k = 0; k < SK_BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) put(cur ^ 1, ra, rb);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int p = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (p >= P) continue;
        float* row = out + (size_t)p * ldg + j0;
        *reinterpret_cast<float4*>(row + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(row + 64 + tx * 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
}

// Gm[p][j] = sum_z parts[z][p][j] in z order (j < ldg; the padding columns are zero in every part)
__global__ void gm_reduce_kernel(const float* __restrict__ parts, int ks, int64_t n, float* __restrict__ Gm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.0f;
    for (int z = 0; z < ks; ++z) v += parts[(size_t)z * n + i];
    Gm[i] = v;
}

// Device workspace of one call (allocated per call: this is a set-up
// routine, not part of the sum).  The GEMM stores whole 128-column blocks,
// so the Gram rows (ldc) and the gradient rows (ldg) are padded to 128.
struct DesignWork {
    float *C = nullptr, *T = nullptr, *Gm = nullptr, *r = nullptr, *m = nullptr, *v = nullptr;
    float* parts = nullptr;  // split-K partials of Gm (ks x P x ldg)
    double* e = nullptr;
    int64_t ldc = 0, ldg = 0, kc = 0;
    int ks = 1;
    ~DesignWork()
    {
        cudaFree(parts);
        cudaFree(C);
        cudaFree(T);
        cudaFree(Gm);
        cudaFree(r);
        cudaFree(m);
        cudaFree(v);
        cudaFree(e);
    }
    cudaError_t alloc(int d, int P, bool adam)
    {
        ldc = ((int64_t)P + 127) / 128 * 128;
        ldg = ((int64_t)d + 127) / 128 * 128;
        cudaError_t err = cudaMalloc(&C, sizeof(float) * (size_t)P * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&T, sizeof(float) * (size_t)d * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&Gm, sizeof(float) * (size_t)P * ldg);
        if (err == cudaSuccess) err = cudaMalloc(&r, sizeof(float) * (size_t)P);
        if (err == cudaSuccess) err = cudaMalloc(&e, sizeof(double) * (size_t)P);
        if (adam && err == cudaSuccess) err = cudaMalloc(&m, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMalloc(&v, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMemset(m, 0, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMemset(v, 0, sizeof(float) * (size_t)P * d);
        // split the inner length of the second contraction into ks ranges (multiples of the
        // slab depth, at least 256 long, at most 20) so that tiles x ks CTAs fill whole waves
        // of the resident CTAs as nearly as possible (fewer ranges on a tie)
        const int64_t tiles = (((int64_t)P + 127) / 128) * (ldg / 128);
        int dev = 0, sms = 1, occ = 1;
        if (err == cudaSuccess) err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gm_splitk_kernel, 256, 0);
        const int64_t resident = (int64_t)sms * (occ > 0 ? occ : 1);
        ks = 1;
        double best = -1.0;
        for (int k = 1; k <= 20 && (k == 1 || ldc / k >= 256); ++k) {
            const int64_t ctas = tiles * k;
            const double eff = (double)ctas / (double)(((ctas + resident - 1) / resident) * resident);
            if (eff > best + 1e-9) {
                best = eff;
                ks = k;
            }
        }
        kc = ((ldc + ks - 1) / ks + 7) / 8 * 8;
        ks = (int)((ldc + kc - 1) / kc);
        if (ks > 1 && err == cudaSuccess) err = cudaMalloc(&parts, sizeof(float) * (size_t)ks * P * ldg);
        return err;
    }
};

// Energy terms and the gradient pieces (r, Gm) of the rows in xi.
cudaError_t esym_pieces(const float* xi, int d, int P, DesignWork& w, cudaStream_t st, bool energy)
{
    cudaError_t e = qs_launch_project_fp32(xi, P, d, xi, P, w.C, w.ldc, st);  // C = Xi Xi^T
    if (e != cudaSuccess) return e;
    if (energy) esym_weights_kernel<true><<<P, 256, 0, st>>>(w.C, P, w.ldc, w.r, w.e);
    else esym_weights_kernel<false><<<P, 256, 0, st>>>(w.C, P, w.ldc, w.r, w.e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 tg((unsigned)((w.ldc + 31) / 32), (unsigned)((d + 31) / 32));
    transpose_pad_kernel<<<tg, dim3(32, 8), 0, st>>>(xi, P, d, w.ldc, w.T);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Gm[p][j] = sum_q W[p][q] Xi[q][j]: rows of W against rows of Xi^T, inner length ldc
    if (w.ks <= 1) return qs_launch_project_fp32(w.T, d, (int)w.ldc, w.C, P, w.Gm, w.ldg, st);
    dim3 g((unsigned)((P + SK_BM - 1) / SK_BM), (unsigned)(w.ldg / SK_BN), (unsigned)w.ks);
    gm_splitk_kernel<<<g, 256, 0, st>>>(w.C, P, w.ldc, w.T, d, w.kc, w.parts, w.ldg);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)P * w.ldg;
    gm_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.parts, w.ks, n, w.Gm);
    return cudaGetLastError();
}

qs_status sum_energy(const DesignWork& w, int P, cudaStream_t st, double* energy)
{
    std::vector<double> e(P);
    if (cudaMemcpyAsync(e.data(), w.e, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return QS_ERR_CUDA;
    double tot = 0.0;
    for (int p = 0; p < P; ++p) tot += e[p];  // fixed order
    *energy = -2.0 * tot;
    return QS_OK;
}

qs_status design_args(const float* dirs, int d, int P)
{
    if (!dirs || d < 1 || P < 1) return QS_ERR_ARG;
    if ((int64_t)P * (((int64_t)P + 127) / 128 * 128) > ((int64_t)1 << 31)) return QS_ERR_UNSUPPORTED;
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_distance_energy(const float* dirs_dev, int d, int P, double* energy, float* grad_dev,
                                        void* stream)
{
    qs_status s = design_args(dirs_dev, d, P);
    if (s == QS_ERR_ARG) return design_fail(QS_ERR_ARG, "qs_distance_energy: bad arguments");
    if (s != QS_OK) return design_fail(s, "qs_distance_energy: P too large (P^2 floats of workspace)");
    cudaStream_t st = (cudaStream_t)stream;
    DesignWork w;
    cudaError_t e = w.alloc(d, P, false);
    if (e != cudaSuccess) return design_fail(QS_ERR_OOM, "qs_distance_energy: workspace allocation failed");
    e = esym_pieces(dirs_dev, d, P, w, st, true);
    if (e == cudaSuccess && grad_dev) {
        // m == NULL: the kernel only reads xi and writes the gradient
        esym_step_kernel<<<P, 256, 0, st>>>(const_cast<float*>(dirs_dev), d, w.r, w.Gm, w.ldg, grad_dev, nullptr,
                                            nullptr, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return design_fail(QS_ERR_CUDA, cudaGetErrorString(e));
    double E = 0.0;
    if (sum_energy(w, P, st, &E) != QS_OK) return design_fail(QS_ERR_CUDA, "qs_distance_energy: readback");
    if (energy) *energy = E;
    return QS_OK;
}

extern "C" qs_status qs_distance_design(float* dirs_dev, int d, int P, int iters, double lr, double* energy,
                                        void* stream)
{
    qs_status s = design_args(dirs_dev, d, P);
    if (s == QS_ERR_ARG || iters < 0 || !(lr > 0.0))
        return design_fail(QS_ERR_ARG, "qs_distance_design: bad arguments");
    if (s != QS_OK) return design_fail(s, "qs_distance_design: P too large (P^2 floats of workspace)");
    cudaStream_t st = (cudaStream_t)stream;
    DesignWork w;
    cudaError_t e = w.alloc(d, P, true);
    if (e != cudaSuccess) return design_fail(QS_ERR_OOM, "qs_distance_design: workspace allocation failed");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double b1t = 1.0, b2t = 1.0;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        e = esym_pieces(dirs_dev, d, P, w, st, false);
        if (e != cudaSuccess) break;
        b1t *= b1;
        b2t *= b2;
        // cosine annealing from lr to lr/100: a constant Adam step keeps moving by ~lr on a
        // deterministic objective instead of settling
        const double lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(3.14159265358979323846 * it / iters)));
        esym_step_kernel<<<P, 256, 0, st>>>(dirs_dev, d, w.r, w.Gm, w.ldg, nullptr, w.m, w.v, (float)lr_t, b1, b2,
                                            (float)b1t, (float)b2t, eps);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && energy) e = esym_pieces(dirs_dev, d, P, w, st, true);
    if (e != cudaSuccess) return design_fail(QS_ERR_CUDA, cudaGetErrorString(e));
    if (energy && sum_energy(w, P, st, energy) != QS_OK)
        return design_fail(QS_ERR_CUDA, "qs_distance_design: readback");
    if (!energy && cudaStreamSynchronize(st) != cudaSuccess)
        return design_fail(QS_ERR_CUDA, "qs_distance_design: synchronise");
    return QS_OK;
}
