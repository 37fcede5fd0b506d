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
// i.e. two P x P x d contractions plus elementwise work, both on the
// library's tcgen05 GEMM in BF16x3 (split operands, FP32 accumulation; the
// products carry ~2^-16 relative error).  a_pq would amplify an error in c_pq
// by about a_pq^3 for near-coincident directions (in d = 3 with P = 1000,
// taking 2 - 2c from the split-BF16 Gram moved the gradient by 6.5e-4 of its
// largest entry), so the weights take |xi_p -+ xi_q|^2 from the rows for
// |c| > 1/2 (esym_weights_kernel).
#include <cuda_bf16.h>
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

// Row p of the Gram matrix C (stride ldc) -> weights W = B - A as the split
// BF16 operands of the second contraction (hi = bf16(W), lo = bf16(W - hi);
// zero in the padding columns P .. ldc-1); r_p; and (ENERGY) the row's share of
// the energy, sum_q (|xi_p - xi_q| + |xi_p + xi_q|), in FP64.  One CTA per row.
// |xi_p -+ xi_q|^2 is 2 -+ 2 c_pq except for near-parallel (c > 1/2) or
// near-antipodal (c < -1/2) pairs, where it is summed from the rows
// themselves: there 1/|xi_p -+ xi_q| would multiply the error of c by up to
// its cube (and 2 -+ 2c cancels), elsewhere the weights change by at most the
// error of c.  The optimiser's steps need no energy: its two FP64 square roots
// per pair would cost about as much as the step's contractions on this GPU's
// FP64 pipe.
template <bool ENERGY>
__global__ void __launch_bounds__(256) esym_weights_kernel(const float* __restrict__ C, int P, int64_t ldc,
                                                           const float* __restrict__ xi, int d,
                                                           __nv_bfloat16* __restrict__ wh,
                                                           __nv_bfloat16* __restrict__ wl,
                                                           float* __restrict__ r, double* __restrict__ e_row)
{
    extern __shared__ float xp[];  // row p of xi
    const int p = blockIdx.x;
    for (int j = threadIdx.x; j < d; j += blockDim.x) xp[j] = xi[(size_t)p * d + j];
    __syncthreads();
    const float* row = C + (size_t)p * ldc;
    __nv_bfloat16* hrow = wh + (size_t)p * ldc;
    __nv_bfloat16* lrow = wl + (size_t)p * ldc;
    float racc = 0.0f;
    double eacc = 0.0;
    // two columns per thread and step (8-byte loads, 4-byte stores of each BF16 pair)
    for (int64_t q0 = 2 * (int64_t)threadIdx.x; q0 < ldc; q0 += 2 * (int64_t)blockDim.x) {
        const float2 c2 = *reinterpret_cast<const float2*>(row + q0);
        float wv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t q = q0 + h;
            wv[h] = 0.0f;
            if (q >= P) continue;
            const float c = fminf(1.0f, fmaxf(-1.0f, h ? c2.y : c2.x));
            float dm2 = 2.0f - 2.0f * c, dp2 = 2.0f + 2.0f * c;
            if (c > 0.5f || c < -0.5f) {
                const float sg = c > 0.0f ? -1.0f : 1.0f;  // xi_p - xi_q or xi_p + xi_q
                const float* xq = xi + (size_t)q * d;
                float s2 = 0.0f;
                for (int j = 0; j < d; ++j) {
                    const float t = fmaf(sg, __ldg(&xq[j]), xp[j]);
                    s2 = fmaf(t, t, s2);
                }
                if (c > 0.0f) dm2 = s2;
                else dp2 = s2;
            }
            // coincident or antipodal pairs have no gradient direction: weight 0
            const float a = (q == p || dm2 <= 0.0f) ? 0.0f : rsqrtf(dm2);
            const float b = dp2 > 0.0f ? rsqrtf(dp2) : 0.0f;
            wv[h] = b - a;
            racc += a + b;
            if (ENERGY) eacc += (q == p ? 0.0 : sqrt((double)dm2)) + sqrt((double)dp2);
        }
        const __nv_bfloat162 hv = __floats2bfloat162_rn(wv[0], wv[1]);
        const float2 hf = __bfloat1622float2(hv);
        *reinterpret_cast<__nv_bfloat162*>(hrow + q0) = hv;
        *reinterpret_cast<__nv_bfloat162*>(lrow + q0) = __floats2bfloat162_rn(wv[0] - hf.x, wv[1] - hf.y);
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

// Gm[p][j] = sum_z parts[z][p][j] in z order (j < ldg; every part covers all of it)
__global__ void gm_reduce_kernel(const float* __restrict__ parts, int ks, int64_t n, float* __restrict__ Gm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.0f;
    for (int z = 0; z < ks; ++z) v += parts[(size_t)z * n + i];
    Gm[i] = v;
}

constexpr int KMAX_SPLITS = 20;
constexpr int TMAP_BYTES = 128;  // sizeof(CUtensorMap)

// Device workspace of one call (allocated per call: this is a set-up
// routine, not part of the sum).  Both contractions run on the tcgen05 GEMM
// in BF16x3 (hi hi + hi lo + lo hi, FP32 accumulation), which computes
// U[p][n] = <A_n, B_p> for rows A_n of its first operand and B_p of its
// second and stores whole 128-row tiles of A:
//   the Gram matrix C = Xi Xi^T      A = B = Xi (K = d), U = C (stride ldc);
//   Gm = (B - A) Xi = W Xi            A = T = Xi^T (d rows), B = W (P rows),
//                                     K = ldc split into ks ranges of kc, one
//                                     GEMM each on its own stream (the d x P
//                                     output has few tiles for its long inner
//                                     length, so one launch would leave most
//                                     SMs idle), whose partial Gm (stride ldg)
//                                     are summed in range order.
// Rows of C and Gm are padded to 128 for the whole-tile stores; the weights
// are zero in the padding columns, so the ranges cover exactly the inner sum.
struct DesignWork {
    float *C = nullptr, *T = nullptr, *Gm = nullptr, *r = nullptr, *m = nullptr, *v = nullptr;
    float* parts = nullptr;  // partial Gm of the inner ranges (ks x P x ldg)
    double* e = nullptr;
    void *xh = nullptr, *xl = nullptr, *wh = nullptr, *wl = nullptr, *th = nullptr, *tl = nullptr;  // BF16 hi / lo
    unsigned int* flag = nullptr;  // the GEMM's timeout flag
    cudaStream_t ss[KMAX_SPLITS] = {};  // one per inner range
    cudaEvent_t fork = nullptr, done[KMAX_SPLITS] = {};
    int64_t ldc = 0, ldg = 0, kc = 0;
    int ldk = 0, ks = 1;
    alignas(64) unsigned char gram_maps[4 * TMAP_BYTES];             // A0 A1 (Xi), B0 B1 (Xi)
    alignas(64) unsigned char gm_maps[KMAX_SPLITS][4 * TMAP_BYTES];  // per range: A0 A1 (T), B0 B1 (W)
    ~DesignWork()
    {
        void* bufs[] = {parts, C, T, Gm, r, m, v, e, xh, xl, wh, wl, th, tl, flag};
        for (void* b : bufs) cudaFree(b);
        for (int z = 0; z < KMAX_SPLITS; ++z) {
            if (ss[z]) cudaStreamDestroy(ss[z]);
            if (done[z]) cudaEventDestroy(done[z]);
        }
        if (fork) cudaEventDestroy(fork);
    }
    cudaError_t alloc(int d, int P, bool adam)
    {
        ldc = ((int64_t)P + 127) / 128 * 128;
        ldg = ((int64_t)d + 127) / 128 * 128;
        ldk = (d + 7) / 8 * 8;
        cudaError_t err = cudaMalloc(&C, sizeof(float) * (size_t)P * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&T, sizeof(float) * (size_t)d * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&Gm, sizeof(float) * (size_t)P * ldg);
        if (err == cudaSuccess) err = cudaMalloc(&r, sizeof(float) * (size_t)P);
        if (err == cudaSuccess) err = cudaMalloc(&e, sizeof(double) * (size_t)P);
        if (err == cudaSuccess) err = cudaMalloc(&xh, 2 * (size_t)P * ldk);
        if (err == cudaSuccess) err = cudaMalloc(&xl, 2 * (size_t)P * ldk);
        if (err == cudaSuccess) err = cudaMalloc(&wh, 2 * (size_t)P * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&wl, 2 * (size_t)P * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&th, 2 * (size_t)d * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&tl, 2 * (size_t)d * ldc);
        if (err == cudaSuccess) err = cudaMalloc(&flag, sizeof(unsigned int));
        if (err == cudaSuccess) err = cudaMemset(flag, 0, sizeof(unsigned int));
        if (adam && err == cudaSuccess) err = cudaMalloc(&m, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMalloc(&v, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMemset(m, 0, sizeof(float) * (size_t)P * d);
        if (adam && err == cudaSuccess) err = cudaMemset(v, 0, sizeof(float) * (size_t)P * d);
        if (err != cudaSuccess) return err;
        // inner ranges of the second contraction: multiples of 64, at least 256 long (unless
        // there is one), at most KMAX_SPLITS, chosen so that the ranges' tiles together fill
        // whole waves of one GEMM CTA per SM as nearly as possible (fewer ranges on a tie)
        int dev = 0, sms = 1;
        err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
        const int64_t tiles = (ldg / 128) * (((int64_t)P + 255) / 256);
        ks = 1;
        kc = ldc;
        double best = -1.0;
        for (int k = 1; k <= KMAX_SPLITS; ++k) {
            const int64_t kck = ((ldc + k - 1) / k + 63) / 64 * 64;
            const int ksk = (int)((ldc + kck - 1) / kck);
            if (ksk > 1 && kck < 256) break;
            const int64_t t = tiles * ksk;
            const double eff = (double)t / (double)(((t + sms - 1) / sms) * sms);
            if (eff > best + 1e-9) {
                best = eff;
                ks = ksk;
                kc = kck;
            }
        }
        if (ks > 1) err = cudaMalloc(&parts, sizeof(float) * (size_t)ks * P * ldg);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int z = 0; z < ks && err == cudaSuccess; ++z) {
            err = cudaStreamCreateWithFlags(&ss[z], cudaStreamNonBlocking);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&done[z], cudaEventDisableTiming);
        }
        if (err != cudaSuccess) return err;
        // tensor maps (K-major BF16 rows; coordinates past a range's end read zeros)
        unsigned char* g = gram_maps;
        bool ok = qs_make_tmap(g + 0 * TMAP_BYTES, xh, 2, d, P, ldk, 128) &&
                  qs_make_tmap(g + 1 * TMAP_BYTES, xl, 2, d, P, ldk, 128) &&
                  qs_make_tmap(g + 2 * TMAP_BYTES, xh, 2, d, P, ldk, 256) &&
                  qs_make_tmap(g + 3 * TMAP_BYTES, xl, 2, d, P, ldk, 256);
        for (int z = 0; ok && z < ks; ++z) {
            const int64_t k0 = (int64_t)z * kc;
            const int klen = (int)(ldc - k0 < kc ? ldc - k0 : kc);
            unsigned char* q = gm_maps[z];
            const size_t off = 2 * (size_t)k0;  // bytes: a multiple of 128
            ok = qs_make_tmap(q + 0 * TMAP_BYTES, (char*)th + off, 2, klen, d, (int)ldc, 128) &&
                 qs_make_tmap(q + 1 * TMAP_BYTES, (char*)tl + off, 2, klen, d, (int)ldc, 128) &&
                 qs_make_tmap(q + 2 * TMAP_BYTES, (char*)wh + off, 2, klen, P, (int)ldc, 256) &&
                 qs_make_tmap(q + 3 * TMAP_BYTES, (char*)wl + off, 2, klen, P, (int)ldc, 256);
        }
        return ok ? cudaSuccess : cudaErrorInvalidValue;
    }
};

// Energy terms and the gradient pieces (r, Gm) of the rows in xi.
cudaError_t esym_pieces(const float* xi, int d, int P, DesignWork& w, cudaStream_t st, bool energy)
{
    // C = Xi Xi^T
    cudaError_t e = qs_launch_split_bf16(xi, P, d, w.ldk, w.xh, w.xl, st);
    if (e == cudaSuccess) e = qs_launch_project_tc(0, w.gram_maps, 0, P, d, P, w.C, w.ldc, w.flag, st, false);
    if (e != cudaSuccess) return e;
    const size_t xs = sizeof(float) * (size_t)d;  // row p in shared memory
    if (xs > 48 * 1024) {
        e = cudaFuncSetAttribute(esym_weights_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(esym_weights_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
        if (e != cudaSuccess) return e;
    }
    __nv_bfloat16* wh = static_cast<__nv_bfloat16*>(w.wh);
    __nv_bfloat16* wl = static_cast<__nv_bfloat16*>(w.wl);
    if (energy) esym_weights_kernel<true><<<P, 256, xs, st>>>(w.C, P, w.ldc, xi, d, wh, wl, w.r, w.e);
    else esym_weights_kernel<false><<<P, 256, xs, st>>>(w.C, P, w.ldc, xi, d, wh, wl, w.r, w.e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 tg((unsigned)((w.ldc + 31) / 32), (unsigned)((d + 31) / 32));
    transpose_pad_kernel<<<tg, dim3(32, 8), 0, st>>>(xi, P, d, w.ldc, w.T);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = qs_launch_split_bf16(w.T, d, (int)w.ldc, (int)w.ldc, w.th, w.tl, st);
    // Gm[p][j] = sum_q W[p][q] T[j][q]: the ranges on their own streams, forked from and
    // joined back into st
    if (e == cudaSuccess) e = cudaEventRecord(w.fork, st);
    for (int z = 0; z < w.ks && e == cudaSuccess; ++z) {
        const int64_t k0 = (int64_t)z * w.kc;
        const int klen = (int)(w.ldc - k0 < w.kc ? w.ldc - k0 : w.kc);
        float* out = w.ks > 1 ? w.parts + (size_t)z * P * w.ldg : w.Gm;
        e = cudaStreamWaitEvent(w.ss[z], w.fork, 0);
        if (e == cudaSuccess) e = qs_launch_project_tc(0, w.gm_maps[z], 0, d, klen, P, out, w.ldg, w.flag, w.ss[z], false);
        if (e == cudaSuccess) e = cudaEventRecord(w.done[z], w.ss[z]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, w.done[z], 0);
    }
    if (e != cudaSuccess || w.ks <= 1) return e;
    const int64_t n = (int64_t)P * w.ldg;
    gm_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.parts, w.ks, n, w.Gm);
    return cudaGetLastError();
}

// The GEMM's timeout flag after the stream has finished (0: none)
bool gemm_timed_out(const DesignWork& w)
{
    unsigned int f = 0;
    return cudaMemcpy(&f, w.flag, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess || f != 0;
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
    if (e != cudaSuccess)
        return design_fail(QS_ERR_OOM, "qs_distance_energy: workspace allocation or tensor-map setup failed");
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
    if (gemm_timed_out(w)) return design_fail(QS_ERR_CUDA, "qs_distance_energy: tensor-core GEMM timed out");
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
    if (e != cudaSuccess)
        return design_fail(QS_ERR_OOM, "qs_distance_design: workspace allocation or tensor-map setup failed");
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
    if (gemm_timed_out(w)) return design_fail(QS_ERR_CUDA, "qs_distance_design: tensor-core GEMM timed out");
    return QS_OK;
}
