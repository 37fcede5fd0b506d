// Grid stages of the sliced fast Fourier summation (arXiv 2410.01316, App. C
// Step 3, eq. 1d_sum_fourier; App. G, eq. Fourier-slicing):
//
//   coefficients  c_k = tau f^(tau k) in FP64 and the filter
//                 D_k = c_k / psi^(k/G)^2                         (Step 2)
//   spread        grid_p[l] = sum_n w_n psi(u_{n,p} - l)          (adjoint NFFT, window part)
//   filter        h_p = IDFT( D . DFT(grid_p) ) restricted to |k| <= N_ft/2
//   interpolate   t_{m,p} = sum_l h_p[l] psi(u_{m,p} - l)         (NFFT, window part)
//   reduce        s_m = (1/P) sum_p t_{m,p}  in a fixed order with TwoSum
//
// The spread writes every point's W taps into a per-slice grid in shared
// memory; the FFT, the filter and the inverse FFT run on the same
// shared-memory grid, so a slice touches HBM only to read its projections and
// to write G filtered values.
//
// The grid is accumulated in 32-bit fixed point with integer shared-memory
// atomics: every cell is bounded by B = sum_n |w_n| (the window is <= 1), so
// with the scale 2^30 / B no sum can overflow, each contribution is rounded
// once to B 2^-31, and integer addition makes the grid independent of the
// order in which threads add.  (FP32 atomicAdd on shared memory is retried
// under contention; the projections of clustered data hit a few hundred cells.)
#include <float.h>
#include <limits.h>
#include <math.h>

#include "qs_device.cuh"
#include "qs_internal.cuh"

using namespace qsdev;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// FP64 Fourier coefficients (App. C Step 2; App. G), one thread per k.
// Gauss:   f^(w) = sqrt(2) pi sigma (2 pi^2 sigma^2 w^2)^{(d-1)/2} e^{-2 pi^2 sigma^2 w^2} / Gamma(d/2)
// Laplace: f^(w) = Gamma((d+1)/2) 2^d pi^{d-1/2} |w|^{d-1} / (Gamma(d/2) alpha^d)
//                  (1 + 4 pi^2 w^2 / alpha^2)^{-(d+1)/2}
// Matern:  f^(w) = Gamma(nu + d/2) 2^{d/2} pi^d beta^d |w|^{d-1}
//                  / (Gamma(d/2) Gamma(nu) nu^{d/2}) (1 + 2 pi^2 beta^2 w^2 / nu)^{-(nu + d/2)}
// All follow from F_1[f](w) = pi^{d/2}/Gamma(d/2) |w|^{d-1} F_d[F](|w|) and
// are evaluated in log space (d up to the hundreds).  Negative distance: the
// 1-periodic triangle wave -(c_d/tau)|t| with closed-form coefficients.
// (Riesz and the thin plate spline come from the host as a table.)
// ---------------------------------------------------------------------------
__device__ double coeff_k(int kernel, double kp, double kp2, int d, double tau, int k)
{
    if (kernel == QS_MATERN) {
        const double w = fabs(tau * (double)k), nu = kp2;
        if (w == 0.0 && d > 1) return 0.0;
        const double lf = lgamma(nu + 0.5 * d) + 0.5 * d * log(2.0) + d * log(kPi) + d * log(kp)
                          + (d > 1 ? (d - 1) * log(w) : 0.0) - lgamma(0.5 * d) - lgamma(nu) - 0.5 * d * log(nu)
                          - (nu + 0.5 * d) * log1p(2.0 * kPi * kPi * kp * kp * w * w / nu);
        return tau * exp(lf);
    }
    if (kernel == QS_NEGDIST) {
        const double cd = exp(0.5 * log(kPi) + lgamma(0.5 * (d + 1)) - lgamma(0.5 * d));
        const double amp = cd / tau;
        if (k == 0) return -0.25 * amp;
        if (k & 1) return amp / (kPi * kPi * (double)k * (double)k);
        return 0.0;
    }
    const double w = fabs(tau * (double)k);
    double lf;
    if (kernel == QS_GAUSS) {
        if (w == 0.0) return d == 1 ? tau * sqrt(2.0 * kPi) * kp : 0.0;
        const double q = 2.0 * kPi * kPi * kp * kp * w * w;
        lf = 0.5 * log(2.0) + log(kPi) + log(kp) + 0.5 * (d - 1) * log(q) - q - lgamma(0.5 * d);
    } else {
        if (w == 0.0) return d == 1 ? tau * 2.0 / kp : 0.0;
        lf = lgamma(0.5 * (d + 1)) + d * log(2.0) + (d - 0.5) * log(kPi) + (d - 1) * log(w)
             - lgamma(0.5 * d) - d * log(kp) - 0.5 * (d + 1) * log1p(4.0 * kPi * kPi * w * w / (kp * kp));
    }
    return tau * exp(lf);
}

// c_in (n_ft values at k + n_ft/2, or NULL): coefficients computed on the host.
__global__ void coeff_kernel(int kernel, double kp, double kp2, int d, double tau, int n_ft, int G,
                             const double* __restrict__ psihat, const double* __restrict__ c_in,
                             double* __restrict__ c_out, float* __restrict__ D_out)
{
    const int K = n_ft / 2;
    const int Gh = G / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    auto ck = [&](int k) {
        if (c_in) return c_in[(k < K ? k : -k) + K];  // c_K = c_{-K} (even)
        return coeff_k(kernel, kp, kp2, d, tau, k);
    };
    if (i < n_ft) c_out[i] = ck(i - K);
    if (i <= Gh) {
        float v = 0.0f;
        if (i <= K) {
            const double ph = psihat[i];
            double dv = ck(i) / (ph * ph);
            // only k = -N_ft/2 is kept of the pair +-N_ft/2; its real part
            // contributes half to each side of the Hermitian spectrum
            if (i == K) dv *= 0.5;
            v = (float)dv;
        }
        D_out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// B = sum_n |w_n| (N if w is NULL) in a fixed order; writes the fixed-point
// scale 2^30 / B and its inverse.  One CTA of 1024 threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) weight_scale_kernel(const float* __restrict__ w, int64_t N,
                                                            float* __restrict__ out, unsigned int* flag)
{
    __shared__ float red[32];
    float acc = 0.0f;
    if (w) {
        for (int64_t n = threadIdx.x; n < N; n += blockDim.x) acc += fabsf(__ldg(&w[n]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) {
            // FP32 summation error is far below the factor-2 headroom of the
            // 2^30 scale (the grid overflows only past 2^31).
            const float B = w ? acc : (float)N;
            float scale = 0.0f, inv = 0.0f;
            if (!isfinite(B)) {
                atomicOr(flag, QS_FLAG_NONFINITE);
            } else if (B > 0.0f) {
                scale = 1073741824.0f / B;
                inv = B / 1073741824.0f;
                if (!isfinite(scale)) {  // B below 2^-98: all weights negligible
                    scale = 0.0f;
                    inv = 0.0f;
                }
            }
            out[0] = scale;
            out[1] = inv;
        }
    }
}

// ---------------------------------------------------------------------------
// Spread + filter: one CTA per slice p.
// ---------------------------------------------------------------------------
// Spread variants (the integer grid makes them bitwise identical): one point
// per thread, W fixed-point contributions each.
//  - SPREAD_COPIES (PARAM copies): W atomics into one of PARAM lane-private
//    grid copies (copy c shifted by 16 c banks), summed at the end.
//  - SPREAD_THREAD (PARAM cells): each thread owns a column of a window of
//    min(PARAM, G) cells (cell t of thread i at t * 256 + i), updated with plain
//    loads and stores, no atomics.  The window is centred on a strided sample of
//    256 of the slice's points; points whose taps leave it use atomics on the
//    one shared grid.  Columns are summed into that grid before the FFT.
// Each grid copy is linear, G + 16 cells, holding cell c at index
// (c + H) mod G with H = G/2 + 8, so the taps of a point at grid coordinate
// u in [-G/2, G/2] fill indices l0 + H .. l0 + H + W - 1, all inside
// [2, G + 14): one base address per point, no wrap-around per tap.  The 16
// overflow cells fold back onto the first 16 before the FFT.  The cyclic
// shift by H commutes with the filter (a cyclic convolution) and is undone
// when the filtered row is stored.
// The spread of a point is short next to the latency of loading its
// projection, so each thread loads PF points at once before spreading them.
enum { SPREAD_COPIES = 0, SPREAD_THREAD = 1 };
constexpr int SPREAD_PAD = QS_SPREAD_PAD;

template <int W, bool FUSED>
__device__ __forceinline__ float spread_u(const qs_launch& L, const float* __restrict__ x, const float* urow,
                                          const float* xi_sm, int64_t n)
{
    float u;
    if (FUSED) {
        const float* xn = x + (size_t)n * L.d;
        u = 0.0f;
        for (int j = 0; j < L.d; ++j) u = fmaf(xi_sm[j], __ldg(&xn[j]), u);
    } else {
        u = __ldg(&urow[n]);
    }
    return u;
}

// One point: validate (rarely taken branch), taps, fixed-point contributions.
template <int W, int TW>
__device__ __forceinline__ void spread_point(const qs_launch& L, float u, float wn, float scale, int H, int* my,
                                             int* mine, int wbase, int wcells)
{
    if (!(fabsf(u) <= L.half_G && fabsf(wn) <= FLT_MAX)) {
        u = qs_check_u(u, L.half_G, L.flag);
        if (!isfinite(wn)) {
            atomicOr(L.flag, QS_FLAG_NONFINITE);
            wn = 0.0f;
        }
    }
    const float ws = wn * scale;
    int l0;
    float tap[W];
    qs_taps<W>(u, L.win, l0, tap);
    const int k0 = l0 + H;
    int q[W];
#pragma unroll
    for (int j = 0; j < W; ++j) q[j] = __float2int_rn(ws * tap[j]);
    if (TW) {
        const unsigned rel = (unsigned)(k0 - wbase);
        if (rel <= (unsigned)(wcells - W)) {
            int* cell = mine + (rel << 8);
#pragma unroll
            for (int j = 0; j < W; ++j) cell[j << 8] += q[j];
            return;
        }
    }
    int* cell = my + k0;
#pragma unroll
    for (int j = 0; j < W; ++j) atomicAdd(&cell[j], q[j]);
}

// Filter the shifted grid of slice p (FFT, c_k / psi^2, inverse FFT) and
// store it unshifted: cell c sits at index (c + H) mod G, H a multiple of 4.
__device__ __forceinline__ void filter_store(const qs_launch& L, float* grid, int p, int H)
{
    const int G = L.G;
    const int Gh = G >> 1;
    const int log2n = 31 - __clz(Gh);
    float2* z = reinterpret_cast<float2*>(grid);
    fft_inplace<false>(z, Gh, log2n, L.tw, G);
    real_filter<false>(z, Gh, L.D, L.tw);
    __syncthreads();
    fft_inplace<true>(z, Gh, log2n, L.tw, G);
    float4* dst = reinterpret_cast<float4*>(L.H + (size_t)p * G);
    const float4* src = reinterpret_cast<const float4*>(grid);
    const int hq = H >> 2, qmask = (G >> 2) - 1;
    for (int i = threadIdx.x; i < (G >> 2); i += blockDim.x) dst[i] = src[(i + hq) & qmask];
}

template <int W, bool FUSED, int MODE, int PARAM, int PF>
__global__ void __launch_bounds__(256) spread_filter_kernel(qs_launch L, const float* __restrict__ x,
                                                            const float* __restrict__ w)
{
    constexpr int COPIES = MODE == SPREAD_COPIES ? PARAM : 1;
    constexpr int TW = MODE == SPREAD_THREAD ? PARAM : 0;
    static_assert(TW == 0 || TW >= W, "the thread window holds a point's taps");
    static_assert(W / 2 + 7 < SPREAD_PAD, "taps stay inside the padded grid");
    extern __shared__ float4 smem4[];
    int* gridi = reinterpret_cast<int*>(smem4);
    float* grid = reinterpret_cast<float*>(smem4);
    __shared__ float xi_sm[QS_FUSED_MAX_D];
    __shared__ int s_lo, s_hi;
    const int p = blockIdx.x;
    const int G = L.G;
    const int H = (G >> 1) + 8;
    const int cstride = G + SPREAD_PAD;
    const int wcells = TW > G ? G : TW;
    int* twin = gridi + cstride;  // SPREAD_THREAD: wcells x 256 ints after the grid
    {
        int4* z4 = reinterpret_cast<int4*>(smem4);
        const int n4 = (COPIES * cstride + wcells * 256) >> 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) z4[i] = make_int4(0, 0, 0, 0);
    }
    if (FUSED) {
        for (int j = threadIdx.x; j < L.d; j += blockDim.x) xi_sm[j] = L.xi_s[(size_t)p * L.d + j];
    }
    if (TW && threadIdx.x == 0) {
        s_lo = INT_MAX;
        s_hi = INT_MIN;
    }
    const float scale = __ldg(&L.wscale[0]);
    const float inv_scale = __ldg(&L.wscale[1]);
    const float* urow = L.U + (size_t)p * L.ldU;
    __syncthreads();

    int wbase = 0;
    if (TW) {
        // first grid index of a strided sample of the slice's points
        int lo = INT_MAX, hi = INT_MIN;
        const int ns = L.N < (int64_t)blockDim.x ? (int)L.N : (int)blockDim.x;
        if ((int)threadIdx.x < ns) {
            const int64_t n = (int64_t)threadIdx.x * L.N / ns;
            float u = spread_u<W, FUSED>(L, x, urow, xi_sm, n);
            if (!(fabsf(u) <= L.half_G)) u = 0.0f;  // recorded by the spread itself
            lo = hi = (int)ceilf(u - (float)(W / 2)) + H;
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((threadIdx.x & 31) == 0 && lo <= hi) {
            atomicMin(&s_lo, lo);
            atomicMax(&s_hi, hi);
        }
        __syncthreads();
        if (s_lo <= s_hi) wbase = ((s_lo + s_hi + W) >> 1) - (wcells >> 1);
        wbase = max(0, min(wbase, cstride - wcells));  // window inside the linear grid
    }

    {
        int* my = gridi + ((threadIdx.x & 31) % COPIES) * cstride;
        int* mine = twin + threadIdx.x;
        // PF points per thread per pass: their loads are all issued before the
        // first of them is spread, so PF loads per thread are in flight.
        int64_t n0 = threadIdx.x;
        for (; n0 + (int64_t)(PF - 1) * blockDim.x < L.N; n0 += (int64_t)PF * blockDim.x) {
            float ub[PF], wb[PF];
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int64_t n = n0 + (int64_t)k * blockDim.x;
                ub[k] = spread_u<W, FUSED>(L, x, urow, xi_sm, n);
                wb[k] = w ? __ldg(&w[n]) : 1.0f;
            }
#pragma unroll
            for (int k = 0; k < PF; ++k) spread_point<W, TW>(L, ub[k], wb[k], scale, H, my, mine, wbase, wcells);
        }
        for (; n0 < L.N; n0 += blockDim.x)
            spread_point<W, TW>(L, spread_u<W, FUSED>(L, x, urow, xi_sm, n0), w ? __ldg(&w[n0]) : 1.0f, scale, H,
                                my, mine, wbase, wcells);
    }
    __syncthreads();
    if (TW) {
        // warp k sums the 256 columns of cells k, k + 8, ...
        const int lane = threadIdx.x & 31;
        for (int t = threadIdx.x >> 5; t < wcells; t += blockDim.x >> 5) {
            const int* row = twin + (t << 8);
            int v = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) v += row[lane + 32 * i];
            v = __reduce_add_sync(0xffffffffu, v);
            if (lane == 0) gridi[wbase + t] += v;  // one warp per grid index
        }
        __syncthreads();
    }
    // sum the copies and fold the overflow cells G .. G + 15 onto 0 .. 15
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
        int v = 0;
#pragma unroll
        for (int c = 0; c < COPIES; ++c) {
            v += gridi[c * cstride + i];
            if (i < SPREAD_PAD) v += gridi[c * cstride + G + i];
        }
        grid[i] = (float)v * inv_scale;
    }
    __syncthreads();
    filter_store(L, grid, p, H);
}

// ---------------------------------------------------------------------------
// Moment spread.  Tap j of a point is the polynomial sum_k a_jk t^k in
// t = 2s in (-1, 1] (s the centred fractional offset of qs_taps), so the
// taps a bin b = l0 of the grid receives from its points follow from the K
// fixed-point moments M_bk = sum_n rn(w_n scale t_n^k): cell b + j gets
// sum_k a_jk M_bk.  Moments 0 and 1 are accumulated as the pair
// rn(ws (1 + t)/2), rn(ws (1 - t)/2), whose sum and difference give them
// exactly: with equal weights a constant basis function would make every
// point's rounding error the same, so that it grows like n instead of sqrt(n).  A point then costs K - 1 products and K conversions
// instead of W polynomial evaluations, and every variant adds the same
// integers into the same bins, so the grids are bitwise identical.  With
// |t| <= 1 each moment stays below 2^30 like a grid cell, and the a_jk of the
// window are below 1 in magnitude (sum_k |a_jk| ~ 1.2), so the quantisation
// error matches that of the tap spread.
// Shared layout: the bin table, (G + 16) bins of K + 1 ints (an odd row
// stride, so random bins spread over the banks), at the bins' linear grid
// indices kb = l0 + H; then, for LW > 0, a window of LW bins with the
// moments of lane i at [bin][k][i] (one bank per lane), centred like the
// thread window of spread_filter_kernel and summed into the table at the
// end; the float grid (G + 16) reuses that space.
// ---------------------------------------------------------------------------
template <int W, int LW>
__device__ __forceinline__ void moment_point(const qs_launch& L, float u, float wn, float scale, int H, int* tab,
                                             int* lanecol, int wbase)
{
    constexpr int m = W / 2;
    constexpr int K = qs_moment_count(W);
    constexpr int KS = K + 1;
    if (!(fabsf(u) <= L.half_G && fabsf(wn) <= FLT_MAX)) {
        u = qs_check_u(u, L.half_G, L.flag);
        if (!isfinite(wn)) {
            atomicOr(L.flag, QS_FLAG_NONFINITE);
            wn = 0.0f;
        }
    }
    const float ws = wn * scale;
    const float fl = ceilf(u - (float)m);
    const int kb = (int)fl + H;
    const float t = 2.0f * ((u - fl) - ((float)m - 0.5f));
    // moments 0 and 1 as ws (1 + t)/2 and ws (1 - t)/2: a basis function
    // constant in t would round every equal weight the same way
    const float hw = 0.5f * ws;
    int q[K];
    q[0] = __float2int_rn(fmaf(hw, t, hw));
    q[1] = __float2int_rn(fmaf(-hw, t, hw));
    float pk = ws * t;
#pragma unroll
    for (int k = 2; k < K; ++k) {
        pk *= t;
        q[k] = __float2int_rn(pk);
    }
    if constexpr (LW > 0) {
        const unsigned rel = (unsigned)(kb - wbase);
        if (rel < (unsigned)LW) {
            int* c = lanecol + rel * (K * 32);
#pragma unroll
            for (int k = 0; k < K; ++k) atomicAdd(&c[k * 32], q[k]);
            return;
        }
    }
    int* c = tab + kb * KS;
#pragma unroll
    for (int k = 0; k < K; ++k) atomicAdd(&c[k], q[k]);
}

// Spread the N points of slice p into moments and turn them into the float
// grid at `grid` (shifted layout, fixed-point scale removed); ends with a
// barrier.  Shared memory as described above.
template <int W, bool FUSED, int LW, int PF>
__device__ __forceinline__ void moment_grid(const qs_launch& L, const float* __restrict__ x,
                                            const float* __restrict__ w, int p, int H, int* tab, float* grid,
                                            const float* xi_sm, int* s_lohi)
{
    constexpr int m = W / 2;
    constexpr int K = qs_moment_count(W);
    constexpr int KS = K + 1;
    constexpr int T = qs_tap_terms(W);
    static_assert(K == 2 * T, "one moment per polynomial coefficient");
    const int G = L.G;
    const int cs = G + SPREAD_PAD;
    int* lanewin = tab + cs * KS;
    const float scale = __ldg(&L.wscale[0]);
    const float inv_scale = __ldg(&L.wscale[1]);
    const float* urow = L.U + (size_t)p * L.ldU;

    int wbase = 0;
    if (LW) {
        int lo = INT_MAX, hi = INT_MIN;
        const int ns = L.N < (int64_t)blockDim.x ? (int)L.N : (int)blockDim.x;
        if ((int)threadIdx.x < ns) {
            const int64_t n = (int64_t)threadIdx.x * L.N / ns;
            float u = spread_u<W, FUSED>(L, x, urow, xi_sm, n);
            if (!(fabsf(u) <= L.half_G)) u = 0.0f;  // recorded by the spread itself
            lo = hi = (int)ceilf(u - (float)m) + H;
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((threadIdx.x & 31) == 0 && lo <= hi) {
            atomicMin(&s_lohi[0], lo);
            atomicMax(&s_lohi[1], hi);
        }
        __syncthreads();
        if (s_lohi[0] <= s_lohi[1]) wbase = ((s_lohi[0] + s_lohi[1]) >> 1) - (LW >> 1);
        wbase = max(0, min(wbase, cs - LW));
    }

    {
        int* lanecol = lanewin + (threadIdx.x & 31);
        // full batches of PF points, software-pipelined: the next batch's
        // loads are in flight while the current one is spread
        const int64_t step = (int64_t)PF * blockDim.x;
        int64_t n0 = threadIdx.x;
        bool have = n0 + (int64_t)(PF - 1) * blockDim.x < L.N;
        float ub[PF], wb[PF];
        if (have) {
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int64_t n = n0 + (int64_t)k * blockDim.x;
                ub[k] = spread_u<W, FUSED>(L, x, urow, xi_sm, n);
                wb[k] = w ? __ldg(&w[n]) : 1.0f;
            }
        }
        while (have) {
            const int64_t n1 = n0 + step;
            const bool next = n1 + (int64_t)(PF - 1) * blockDim.x < L.N;
            float un[PF], wn[PF];
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int64_t n = n1 + (int64_t)k * blockDim.x;
                un[k] = next ? spread_u<W, FUSED>(L, x, urow, xi_sm, n) : 0.0f;
                wn[k] = next ? (w ? __ldg(&w[n]) : 1.0f) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < PF; ++k) moment_point<W, LW>(L, ub[k], wb[k], scale, H, tab, lanecol, wbase);
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                ub[k] = un[k];
                wb[k] = wn[k];
            }
            n0 = n1;
            have = next;
        }
        for (; n0 < L.N; n0 += blockDim.x)
            moment_point<W, LW>(L, spread_u<W, FUSED>(L, x, urow, xi_sm, n0), w ? __ldg(&w[n0]) : 1.0f, scale, H,
                                tab, lanecol, wbase);
    }
    __syncthreads();
    if (LW) {
        // one warp per (bin, moment): sum the 32 lane columns into the table
        const int lane = threadIdx.x & 31;
        for (int r = threadIdx.x >> 5; r < LW * K; r += blockDim.x >> 5) {
            int v = __reduce_add_sync(0xffffffffu, lanewin[r * 32 + lane]);
            if (lane == 0) tab[(wbase + r / K) * KS + r % K] += v;
        }
        __syncthreads();
    }
    // per bin: the W tap sums V_bj = sum_k a_jk M_bk, written over the moments
    // (K >= W); mirrored taps share the even and odd parts
    float* vtab = reinterpret_cast<float*>(tab);
    for (int b = threadIdx.x; b < cs; b += blockDim.x) {
        int* row = tab + b * KS;
        int mk[K];
        bool any = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            mk[k] = row[k];
            any |= mk[k] != 0;
        }
        if (!any) continue;  // the row already reads as W zero floats
        float mh[K];
        mh[0] = (float)(mk[0] + mk[1]);
        mh[1] = 0.5f * (float)(mk[0] - mk[1]);
#pragma unroll
        for (int k = 2; k < K; ++k) mh[k] = ldexpf((float)mk[k], -k);
#pragma unroll
        for (int j = 0; j < m; ++j) {
            float e = 0.0f, o = 0.0f;
#pragma unroll
            for (int i = 0; i < T; ++i) {
                e = fmaf(L.win.e[j][i], mh[2 * i], e);
                o = fmaf(L.win.o[j][i], mh[2 * i + 1], o);
            }
            vtab[b * KS + j] = e + o;
            vtab[b * KS + W - 1 - j] = e - o;
        }
    }
    __syncthreads();
    // cell c = sum_j V_{c-j, j}; the overflow cells G .. G + 15 fold onto 0 .. 15
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (c - j >= 0) v += vtab[(c - j) * KS + j];
        if (c < SPREAD_PAD) {
            float f = 0.0f;
#pragma unroll
            for (int j = 0; j < W; ++j) f += vtab[(G + c - j) * KS + j];
            v += f;
        }
        grid[c] = v * inv_scale;
    }
    __syncthreads();
}

template <int W, bool FUSED, int LW, int PF>
__global__ void __launch_bounds__(512, 2) spread_moment_kernel(qs_launch L, const float* __restrict__ x,
                                                               const float* __restrict__ w)
{
    constexpr int K = qs_moment_count(W);
    extern __shared__ float4 smem4[];
    int* tab = reinterpret_cast<int*>(smem4);
    __shared__ float xi_sm[QS_FUSED_MAX_D];
    __shared__ int s_lohi[2];
    const int p = blockIdx.x;
    const int G = L.G;
    const int H = (G >> 1) + 8;
    const int cs = G + SPREAD_PAD;
    float* grid = reinterpret_cast<float*>(tab + cs * (K + 1));
    {
        int4* z4 = reinterpret_cast<int4*>(smem4);
        const int n4 = (cs * (K + 1) + LW * K * 32) >> 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) z4[i] = make_int4(0, 0, 0, 0);
    }
    if (FUSED)
        for (int j = threadIdx.x; j < L.d; j += blockDim.x) xi_sm[j] = L.xi_s[(size_t)p * L.d + j];
    if (threadIdx.x == 0) {
        s_lohi[0] = INT_MAX;
        s_lohi[1] = INT_MIN;
    }
    __syncthreads();
    moment_grid<W, FUSED, LW, PF>(L, x, w, p, H, tab, grid, xi_sm, s_lohi);
    filter_store(L, grid, p, H);
}

// ---------------------------------------------------------------------------
// Spread for the gradients (fused projection, d <= QS_GRAD_MAX_D), one CTA per slice.
// MODE 1: H2 <- derivative filter (table Dd).  MODE 2: L.H <- plain filter
// (table L.D) and H2 <- derivative filter from the same spread grid.
// ---------------------------------------------------------------------------
// Filter the shifted grid of slice p for the gradients and store unshifted.
// MODE 1: H2 <- derivative filter (table Dd).  MODE 2: also L.H <- plain
// filter, from a copy of the spectrum in grid2.
template <int MODE>
__device__ __forceinline__ void grad_filter_store(const qs_launch& L, float* grid, float* grid2, const float* Dd,
                                                  float* H2, int p, int H)
{
    const int G = L.G;
    const int Gh = G >> 1;
    const int log2n = 31 - __clz(Gh);
    float2* z = reinterpret_cast<float2*>(grid);
    float2* z2 = reinterpret_cast<float2*>(grid2);
    const int hq = H >> 2, qmask = (G >> 2) - 1;
    fft_inplace<false>(z, Gh, log2n, L.tw, G);
    if (MODE == 2) {
        for (int i = threadIdx.x; i < Gh; i += blockDim.x) z2[i] = z[i];
        __syncthreads();
        real_filter<false>(z, Gh, L.D, L.tw);
        real_filter<true>(z2, Gh, Dd, L.tw);
        __syncthreads();
        fft_inplace<true>(z, Gh, log2n, L.tw, G);
        fft_inplace<true>(z2, Gh, log2n, L.tw, G);
        float4* dst = reinterpret_cast<float4*>(L.H + (size_t)p * G);
        const float4* src = reinterpret_cast<const float4*>(grid);
        for (int i = threadIdx.x; i < (G >> 2); i += blockDim.x) dst[i] = src[(i + hq) & qmask];
        float4* dst2 = reinterpret_cast<float4*>(H2 + (size_t)p * G);
        const float4* src2 = reinterpret_cast<const float4*>(grid2);
        for (int i = threadIdx.x; i < (G >> 2); i += blockDim.x) dst2[i] = src2[(i + hq) & qmask];
    } else {
        real_filter<true>(z, Gh, Dd, L.tw);
        __syncthreads();
        fft_inplace<true>(z, Gh, log2n, L.tw, G);
        float4* dst2 = reinterpret_cast<float4*>(H2 + (size_t)p * G);
        const float4* src = reinterpret_cast<const float4*>(grid);
        for (int i = threadIdx.x; i < (G >> 2); i += blockDim.x) dst2[i] = src[(i + hq) & qmask];
    }
}

template <int W, int MODE, bool FUSED>
__global__ void __launch_bounds__(256) spread_grad_kernel(qs_launch L, const float* __restrict__ x,
                                                          const float* __restrict__ w, const float* __restrict__ Dd,
                                                          float* __restrict__ H2)
{
    // same shifted, padded linear grid as spread_filter_kernel (one copy)
    extern __shared__ float4 smem4[];
    int* gridi = reinterpret_cast<int*>(smem4);
    float* grid = reinterpret_cast<float*>(smem4);
    float* grid2 = grid + L.G + SPREAD_PAD;
    __shared__ float xi_sm[QS_FUSED_MAX_D];
    const int p = blockIdx.x;
    const int G = L.G;
    const int H = (G >> 1) + 8;
    for (int i = threadIdx.x; i < G + SPREAD_PAD; i += blockDim.x) gridi[i] = 0;
    if (FUSED)
        for (int j = threadIdx.x; j < L.d; j += blockDim.x) xi_sm[j] = L.xi_s[(size_t)p * L.d + j];
    const float scale = __ldg(&L.wscale[0]);
    const float inv_scale = __ldg(&L.wscale[1]);
    const float* urow = L.U + (size_t)p * L.ldU;
    __syncthreads();
    for (int64_t n = threadIdx.x; n < L.N; n += blockDim.x)
        spread_point<W, 0>(L, spread_u<W, FUSED>(L, x, urow, xi_sm, n), w ? __ldg(&w[n]) : 1.0f, scale, H, gridi,
                           nullptr, 0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
        const int v = gridi[i] + (i < SPREAD_PAD ? gridi[G + i] : 0);
        grid[i] = (float)v * inv_scale;
    }
    __syncthreads();
    grad_filter_store<MODE>(L, grid, grid2, Dd, H2, p, H);
}

// The same from a moment spread (plans whose sums use the moment family, so
// that the plain grid of MODE 2 equals that of spread_moment_kernel bit for bit).
template <int W, int MODE, bool FUSED>
__global__ void __launch_bounds__(512, 2) spread_grad_moment_kernel(qs_launch L, const float* __restrict__ x,
                                                                    const float* __restrict__ w,
                                                                    const float* __restrict__ Dd,
                                                                    float* __restrict__ H2)
{
    constexpr int K = qs_moment_count(W);
    extern __shared__ float4 smem4[];
    int* tab = reinterpret_cast<int*>(smem4);
    __shared__ float xi_sm[QS_FUSED_MAX_D];
    __shared__ int s_lohi[2];
    const int p = blockIdx.x;
    const int G = L.G;
    const int H = (G >> 1) + 8;
    const int cs = G + SPREAD_PAD;
    float* grid = reinterpret_cast<float*>(tab + cs * (K + 1));
    float* grid2 = grid + cs;
    {
        int4* z4 = reinterpret_cast<int4*>(smem4);
        const int n4 = (cs * (K + 1)) >> 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) z4[i] = make_int4(0, 0, 0, 0);
    }
    if (FUSED)
        for (int j = threadIdx.x; j < L.d; j += blockDim.x) xi_sm[j] = L.xi_s[(size_t)p * L.d + j];
    __syncthreads();
    moment_grid<W, FUSED, 0, 4>(L, x, w, p, H, tab, grid, xi_sm, s_lohi);
    grad_filter_store<MODE>(L, grid, grid2, Dd, H2, p, H);
}

// ---------------------------------------------------------------------------
// Derivative interpolation + back-projection (fused projection, d <= DMAX):
//   q_{m,p} = sum_l h'_p[l] psi(u_{m,p} - l),  acc_m += q_{m,p} xi_p
// per slice group, compensated per component.  part: [2][S][M][d].
// ---------------------------------------------------------------------------
template <int W, int DMAX, bool FUSED>
__global__ void __launch_bounds__(256) interp_grad_kernel(qs_launch L, const float* __restrict__ y,
                                                          const float* __restrict__ Hd, const float* __restrict__ xi,
                                                          float* __restrict__ part)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    const int S = gridDim.y;
    if (m >= L.M) return;
    const int d = L.d;
    const int p0 = (int)(((int64_t)g * L.P) / S);
    const int p1 = (int)(((int64_t)(g + 1) * L.P) / S);
    float yr[FUSED ? DMAX : 1], hi[DMAX], lo[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (FUSED) yr[j] = j < d ? __ldg(&y[(size_t)m * d + j]) : 0.0f;
        hi[j] = 0.0f;
        lo[j] = 0.0f;
    }
    const int mask = L.G - 1;
    for (int p = p0; p < p1; ++p) {
        float u;
        if (FUSED) {
            const float* xs = L.xi_s + (size_t)p * d;
            u = 0.0f;
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
                if (j < d) u = fmaf(__ldg(&xs[j]), yr[j], u);
        } else {
            u = __ldg(&L.U[(size_t)p * L.ldU + m]);
        }
        u = qs_check_u(u, L.half_G, L.flag);
        int l0;
        float tap[W];
        qs_taps<W>(u, L.win, l0, tap);
        const float* h = Hd + (size_t)p * L.G;
        float q = 0.0f;
#pragma unroll
        for (int j = 0; j < W; ++j) q = fmaf(__ldg(&h[(l0 + j) & mask]), tap[j], q);
        const float* xp = xi + (size_t)p * d;
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < d) qs_two_sum(hi[j], lo[j], q * __ldg(&xp[j]));
    }
    float* ph = part + ((size_t)g * L.M + m) * d;
    float* pl = part + ((size_t)(S + g) * L.M + m) * d;
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
        if (j < d) {
            ph[j] = hi[j];
            pl[j] = lo[j];
        }
}

// ---------------------------------------------------------------------------
// Gradients for d > QS_GRAD_MAX_D (unfused projection forms): the derivative
// interpolation without the back-projection, written over the projections,
//   q_{m,p} = sum_l h'_p[l] psi(u_{m,p} - l)   in place of u_{m,p} in U,
// then the back-projection onto the directions as a GEMM (backproj_kernel).
// grid (ceil(M / (256 ID_TPT)), P): the CTA stages its slice's derivative row
// once (wrapped by ROW_PAD cells) and walks ID_TPT targets per thread.  The
// taps and their sum are those of interp_grad_kernel, so q is the same number.
// ---------------------------------------------------------------------------
constexpr int ID_TPT = 16;

template <int W>
__global__ void __launch_bounds__(256) interp_deriv_kernel(qs_launch L, const float* __restrict__ Hd)
{
    extern __shared__ float4 drow4[];
    float* row = reinterpret_cast<float*>(drow4);
    const int G = L.G, mask = G - 1;
    const int p = blockIdx.y;
    const float* src = Hd + (size_t)p * G;
    for (int i = threadIdx.x; i < G + ROW_PAD; i += blockDim.x) row[i] = __ldg(&src[i < G ? i : i - G]);
    __syncthreads();
    float* urow = L.U + (size_t)p * L.ldU;
    const int64_t m0 = (int64_t)blockIdx.x * blockDim.x * ID_TPT + threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < ID_TPT; ++i) {
        const int64_t m = m0 + (int64_t)i * blockDim.x;
        if (m >= L.M) break;
        const float u = qs_check_u(urow[m], L.half_G, L.flag);
        int l0;
        float tap[W];
        qs_taps<W>(u, L.win, l0, tap);
        const float* h = row + (l0 & mask);
        float q = 0.0f;
#pragma unroll
        for (int j = 0; j < W; ++j) q = fmaf(h[j], tap[j], q);
        urow[m] = q;
    }
}

// out[m][j] = scale * fac_m * sum_p Q[p][m] xi[p][j] for m < M, j < d: the
// back-projection onto the directions as a GEMM (M x P)(P x d), Q slice-major
// with row stride ldQ, xi P x d row-major.  CTA tile: BP_TM targets x TN
// components (TN = 16, 32 or 64, the smallest covering d up to 64), 256
// threads with RM x 4 outputs each; the slices go in chunks of 16 staged in
// shared memory (both operands coalesced, the next chunk fetched into
// registers during the current one), each chunk's products
// summed by FMA in slice order and the chunk sums accumulated by TwoSum, so
// the result does not depend on the tiling and is reproducible.
constexpr int BP_TK = 16;

template <int TN, int RM>
__global__ void __launch_bounds__(256) backproj_kernel(const float* __restrict__ Q, int64_t ldQ, int64_t M, int P,
                                                       const float* __restrict__ xi, int d, float scale,
                                                       const float* __restrict__ fac, float* __restrict__ out)
{
    constexpr int GX = TN / 4, BP_TN = TN, BP_TM = RM * 256 / GX;
    constexpr int NA = BP_TK * BP_TM / 256, NB = (BP_TK * BP_TN + 255) / 256;  // operand elements per thread
    __shared__ __align__(16) float As[BP_TK][BP_TM];
    __shared__ __align__(16) float Bs[BP_TK][BP_TN];
    const int64_t m0 = (int64_t)blockIdx.x * BP_TM;
    const int j0 = blockIdx.y * BP_TN;
    const int tx = threadIdx.x % GX;  // components j0 + 4 tx .. + 3
    const int ty = threadIdx.x / GX;  // targets m0 + RM ty .. + RM - 1
    float hi[RM][4], lo[RM][4];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) hi[i][k] = lo[i][k] = 0.0f;
    // the next chunk's operands are fetched into registers while the current one is used
    float pa[NA], pb[NB];
    auto fetch = [&](int p0) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int i = threadIdx.x + 256 * q, r = i / BP_TM, c = i - r * BP_TM;
            const int64_t m = m0 + c;
            pa[q] = (p0 + r < P && m < M) ? __ldg(&Q[(size_t)(p0 + r) * ldQ + m]) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int i = threadIdx.x + 256 * q, r = i / BP_TN, c = i - r * BP_TN;
            pb[q] = (i < BP_TK * BP_TN && p0 + r < P && j0 + c < d) ? __ldg(&xi[(size_t)(p0 + r) * d + j0 + c]) : 0.0f;
        }
    };
    fetch(0);
    for (int p0 = 0; p0 < P; p0 += BP_TK) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int i = threadIdx.x + 256 * q, r = i / BP_TM;
            As[r][i - r * BP_TM] = pa[q];
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int i = threadIdx.x + 256 * q, r = i / BP_TN;
            if (i < BP_TK * BP_TN) Bs[r][i - r * BP_TN] = pb[q];
        }
        __syncthreads();
        if (p0 + BP_TK < P) fetch(p0 + BP_TK);
        float acc[RM][4];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = 0.0f;
#pragma unroll 4
        for (int r = 0; r < BP_TK; ++r) {
            float a[RM];
#pragma unroll
            for (int q = 0; q < RM; q += 4) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[r][RM * ty + q]);
                a[q] = a4.x;
                a[q + 1] = a4.y;
                a[q + 2] = a4.z;
                a[q + 3] = a4.w;
            }
            const float4 b = *reinterpret_cast<const float4*>(&Bs[r][4 * tx]);
            const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(a[i], bb[k], acc[i][k]);
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) qs_two_sum(hi[i][k], lo[i][k], acc[i][k]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int64_t m = m0 + RM * ty + i;
        if (m >= M) break;
        const float f = scale * (fac ? __ldg(&fac[m]) : 1.0f);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = j0 + 4 * tx + k;
            if (j < d) out[(size_t)m * d + j] = (hi[i][k] + lo[i][k]) * f;
        }
    }
}

// g[m][j] = scale * fac_m * sum over slice groups (in order) of the partials.
__global__ void reduce_grad_kernel(const float* __restrict__ part, int S, int64_t M, int d, float scale,
                                   const float* __restrict__ fac, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * d) return;
    const int64_t m = i / d;
    float hi = 0.0f, lo = 0.0f;
    for (int g = 0; g < S; ++g) {
        qs_two_sum(hi, lo, part[(size_t)g * M * d + i]);
        lo += part[(size_t)(S + g) * M * d + i];
    }
    const float f = fac ? __ldg(&fac[m]) : 1.0f;
    out[i] = (hi + lo) * scale * f;
}

// Derivative filter table: g_k = 2 pi k c_k / psi^(k/G)^2 for 0 <= k <= N_ft/2
// (half weight at k = N_ft/2, as for the plain filter), 0 beyond.
__global__ void deriv_table_kernel(const double* __restrict__ c, const double* __restrict__ psihat, int n_ft, int G,
                                   float* __restrict__ Dd)
{
    const int K = n_ft / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > G / 2) return;
    float v = 0.0f;
    if (i <= K) {
        const double ck = i < K ? c[i + K] : c[0];  // c_{N_ft/2} = c_{-N_ft/2} (even)
        const double ph = psihat[i];
        double dv = 2.0 * kPi * (double)i * ck / (ph * ph);
        if (i == K) dv *= 0.5;
        v = (float)dv;
    }
    Dd[i] = v;
}

// ---------------------------------------------------------------------------
// Interpolation + per-group compensated slice sums.
// grid: (ceil((m_end - m_base) / (256 TPT)), S); CTA (bx, g) handles the
// targets m_base + bx*256*TPT + i*256 + tid (i < TPT) below m_end and the
// slices [g P / S, (g+1) P / S) in increasing order.  The filtered row of each slice is staged in shared
// memory (double-buffered cp.async) with its first cells repeated after the
// end, so the W taps of a target are read without wrapping.
// ---------------------------------------------------------------------------
// Interpolation of the filtered rows at the targets, per slice group.  Per
// slice, the CTA first locates its targets' bins; when they span fewer than
// QWIN bins (clustered projections) it expands the row into the bins'
// polynomials in t (the tap polynomials of qs_taps summed against the row),
// and each target is one degree-(K-1) Horner evaluation; otherwise each
// target takes its W taps from the row, and the CTA stops looking for
// narrow ranges in its remaining slices.  Both evaluate the same polynomial
// sum_j h[l0 + j] tap_j, rounded differently; which one a target takes
// depends only on the data and the CTA's targets, so results are
// reproducible.  With TPT even, targets go in pairs through packed FP32x2
// arithmetic (each lane rounding as the scalar form).  The block's bin range
// per slice comes from one shared atomic min / max per warp.
constexpr int QWIN = 256;

template <int W, bool FUSED, int DMAX, int TPT>
__global__ void __launch_bounds__(IT_THREADS) interp_kernel(qs_launch L, const float* __restrict__ y)
{
    extern __shared__ float4 rows4[];
    float* rows = reinterpret_cast<float*>(rows4);
    const int G = L.G;
    // per buffer: the filtered row (G + ROW_PAD cells) and, unfused, the
    // projections of the CTA's 256 TPT targets on that slice
    constexpr int UCNT = FUSED ? 0 : IT_THREADS * TPT;
    const int stride = G + ROW_PAD + UCNT;
    const int g = blockIdx.y;
    const int S = gridDim.y;
    const int p0 = (int)(((int64_t)g * L.P) / S);
    const int p1 = (int)(((int64_t)(g + 1) * L.P) / S);
    const int64_t m0 = L.m_base + (int64_t)blockIdx.x * IT_THREADS * TPT;
    const int mask = G - 1;

    // windowed coefficient path: a_jk of tap_j(t) = sum_k a_jk t^k (t = 2 s;
    // from the even / odd tap polynomials), the bins' polynomials Q, the
    // block's bin range
    constexpr int KQ = qs_moment_count(W);
    const int H0 = (G >> 1) + W / 2;
    __shared__ float qwin[KQ * QWIN];
    __shared__ int s_krange[2][2];  // per slice parity: block-wide [min, max] bin
    if (threadIdx.x < 2) {
        s_krange[threadIdx.x][0] = INT_MAX;
        s_krange[threadIdx.x][1] = INT_MIN;
    }  // first read after the loop's first barrier

    float yr[FUSED ? DMAX * TPT : 1];
    float hi[TPT], lo[TPT];
    bool live[TPT];
    bool try_win = true;  // uniform over the block: decided from block-wide values
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
        const int64_t m = m0 + threadIdx.x + (int64_t)i * IT_THREADS;
        live[i] = m < L.m_end;
        hi[i] = 0.0f;
        lo[i] = 0.0f;
        if (FUSED) {
#pragma unroll
            for (int j = 0; j < DMAX; ++j) yr[i * DMAX + j] = (live[i] && j < L.d) ? __ldg(&y[(size_t)m * L.d + j]) : 0.0f;
        }
    }
    // stage slice p: its filtered row and (unfused) the block's projections;
    // a projection chunk is copied only if it lies inside the U row
    auto stage = [&](int p, float* buf) {
        const int n16 = (G + ROW_PAD) >> 2;
        const float* src = L.H + (size_t)p * G;
        for (int i = threadIdx.x; i < n16; i += IT_THREADS) {
            const int c = (i << 2) < G ? (i << 2) : (i << 2) - G;
            cp_async16(buf + (i << 2), src + c);
        }
        if (!FUSED) {
            const float* urow = L.U + (size_t)p * L.ldU + m0;
            for (int i = threadIdx.x; i < UCNT / 4; i += IT_THREADS)
                if (m0 + 4 * i + 3 < L.ldU) cp_async16(buf + G + ROW_PAD + 4 * i, urow + 4 * i);
        }
        cp_async_commit();
    };
    if (p0 < p1) stage(p0, rows);
    for (int p = p0; p < p1; ++p) {
        const float* row = rows + ((p - p0) & 1) * stride;
        if (p + 1 < p1) {
            stage(p + 1, rows + ((p + 1 - p0) & 1) * stride);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (!try_win) {
            // an earlier slice's targets spanned too many bins: taps directly
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                if (!live[i]) continue;
                float u;
                if (FUSED) {
                    const float* xs = L.xi_s + (size_t)p * L.d;
                    u = 0.0f;
#pragma unroll
                    for (int j = 0; j < DMAX; ++j)
                        if (j < L.d) u = fmaf(__ldg(&xs[j]), yr[i * DMAX + j], u);
                } else {
                    u = row[G + ROW_PAD + threadIdx.x + i * IT_THREADS];
                }
                u = qs_check_u(u, L.half_G, L.flag);
                int l0;
                float tap[W];
                qs_taps<W>(u, L.win, l0, tap);
                const float* h = row + (l0 & mask);
                float t = 0.0f;
#pragma unroll
                for (int j = 0; j < W; ++j) t = fmaf(h[j], tap[j], t);
                qs_two_sum(hi[i], lo[i], t);
            }
            __syncthreads();  // the buffer just read is refilled two slices later
            continue;
        }
        // target positions: u, the bin kb = l0 + H0 in [0, G] (l0 the first
        // tap cell, unwrapped) and t = 2 s in (-1, 1]
        float uu[TPT], tt[TPT];
        int kb[TPT];
        int kmin = INT_MAX, kmax = INT_MIN;
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            float u = 0.0f;
            if (live[i]) {
                if (FUSED) {
                    const float* xs = L.xi_s + (size_t)p * L.d;
#pragma unroll
                    for (int j = 0; j < DMAX; ++j)
                        if (j < L.d) u = fmaf(__ldg(&xs[j]), yr[i * DMAX + j], u);
                } else {
                    u = row[G + ROW_PAD + threadIdx.x + i * IT_THREADS];
                }
                u = qs_check_u(u, L.half_G, L.flag);
            }
            uu[i] = u;
            if constexpr (TPT % 2 != 0) {
                const float fl = ceilf(u - (float)(W / 2));
                kb[i] = (int)fl + H0;
                tt[i] = 2.0f * ((u - fl) - ((float)(W / 2) - 0.5f));
            }
        }
        if constexpr (TPT % 2 == 0) {
            // the same bin and offset in packed pairs: fma(2, u - fl, 1 - W)
            // equals 2 ((u - fl) - (W/2 - 1/2)) exactly (scaling by 2 commutes
            // with rounding)
#pragma unroll
            for (int i = 0; i < TPT; i += 2) {
                const float2 u2 = make_float2(uu[i], uu[i + 1]);
                const float2 a2 = __fadd2_rn(u2, make_float2(-(float)(W / 2), -(float)(W / 2)));
                const float2 fl2 = make_float2(ceilf(a2.x), ceilf(a2.y));
                kb[i] = (int)fl2.x + H0;
                kb[i + 1] = (int)fl2.y + H0;
                const float2 t2 = __ffma2_rn(make_float2(2.0f, 2.0f), qs_sub2(u2, fl2),
                                             make_float2((float)(1 - W), (float)(1 - W)));
                tt[i] = t2.x;
                tt[i + 1] = t2.y;
            }
        }
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            if (live[i]) {
                kmin = min(kmin, kb[i]);
                kmax = max(kmax, kb[i]);
            }
        }
        // block range: one shared atomic pair per warp into this slice's
        // cells; thread 0 resets the other parity's cells, last read in the
        // previous slice (two barriers ago) and next written in the next one
        const int par = (p - p0) & 1;
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&s_krange[par][0], kmin);
            atomicMax(&s_krange[par][1], kmax);
        }
        if (threadIdx.x == 0) {
            s_krange[par ^ 1][0] = INT_MAX;
            s_krange[par ^ 1][1] = INT_MIN;
        }
        __syncthreads();
        kmin = s_krange[par][0];
        kmax = s_krange[par][1];
        if (kmin <= kmax && kmax - kmin < QWIN) {
            // the CTA's targets of this slice fall in few bins: per bin b the
            // polynomial Q_b(t) = sum_j h[b + j] tap_j(t) (coefficients
            // sum_j a_jk h[b + j]), then a target costs a Horner evaluation
            // one thread per bin: its W row cells read once, the tap coefficients
            // a_jk 2^-k taken from the launch parameters as constant operands
            const int nb = kmax - kmin + 1;
            for (int b = threadIdx.x; b < nb; b += IT_THREADS) {
                const int c0 = kmin + b - H0;
                float r[W];
#pragma unroll
                for (int j = 0; j < W; ++j) r[j] = row[(c0 + j) & mask];
#pragma unroll
                for (int k = 0; k < KQ; ++k) {
                    float q = 0.0f;
#pragma unroll
                    for (int j = 0; j < W; ++j) q = fmaf(L.atab[j * KQ + k], r[j], q);
                    qwin[k * QWIN + b] = q;  // coefficient-major: lanes at different bins hit different banks
                }
            }
            __syncthreads();
            if constexpr (TPT % 2 == 0) {
                // two targets per packed FP32x2 Horner step and TwoSum (the
                // same roundings as the scalar loop); a dead target reads
                // bin kmin and is never stored
#pragma unroll
                for (int i = 0; i < TPT; i += 2) {
                    const float* qa = qwin + ((live[i] ? kb[i] : kmin) - kmin);
                    const float* qc = qwin + ((live[i + 1] ? kb[i + 1] : kmin) - kmin);
                    const float2 t2 = make_float2(tt[i], tt[i + 1]);
                    float2 v = make_float2(qa[(KQ - 1) * QWIN], qc[(KQ - 1) * QWIN]);
#pragma unroll
                    for (int k = KQ - 2; k >= 0; --k) v = __ffma2_rn(v, t2, make_float2(qa[k * QWIN], qc[k * QWIN]));
                    float2 h2 = make_float2(hi[i], hi[i + 1]), l2 = make_float2(lo[i], lo[i + 1]);
                    qs_two_sum2(h2, l2, v);
                    hi[i] = h2.x;
                    hi[i + 1] = h2.y;
                    lo[i] = l2.x;
                    lo[i + 1] = l2.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < TPT; ++i) {
                    if (!live[i]) continue;
                    const float* qb = qwin + (kb[i] - kmin);
                    float v = qb[(KQ - 1) * QWIN];
#pragma unroll
                    for (int k = KQ - 2; k >= 0; --k) v = fmaf(v, tt[i], qb[k * QWIN]);
                    qs_two_sum(hi[i], lo[i], v);
                }
            }
        } else {
            if (kmin <= kmax) try_win = false;  // spread-out targets: stay on the tap path
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                if (!live[i]) continue;
                int l0;
                float tap[W];
                qs_taps<W>(uu[i], L.win, l0, tap);
                const float* h = row + (l0 & mask);
                float t = 0.0f;
#pragma unroll
                for (int j = 0; j < W; ++j) t = fmaf(h[j], tap[j], t);
                qs_two_sum(hi[i], lo[i], t);
            }
        }
        __syncthreads();  // the buffer just read is refilled two slices later
    }
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
        if (!live[i]) continue;
        const int64_t m = m0 + threadIdx.x + (int64_t)i * IT_THREADS;
        L.part[(size_t)g * L.M + m] = hi[i];
        L.part[(size_t)(S + g) * L.M + m] = lo[i];
    }
}

// s_m = (1/P) sum over slice groups in increasing order (TwoSum).
__global__ void reduce_kernel(const float* __restrict__ part, int S, int64_t M, int P, float* __restrict__ s)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float hi = 0.0f, lo = 0.0f;
    // groups in increasing order; eight groups' loads are issued together
    int g = 0;
    for (; g + 8 <= S; g += 8) {
        float a[8], b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            a[j] = part[(size_t)(g + j) * M + m];
            b[j] = part[(size_t)(S + g + j) * M + m];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            qs_two_sum(hi, lo, a[j]);
            lo += b[j];
        }
    }
    for (; g < S; ++g) {
        qs_two_sum(hi, lo, part[(size_t)g * M + m]);
        lo += part[(size_t)(S + g) * M + m];
    }
    s[m] = (hi + lo) / (float)P;
}

template <int W, bool FUSED, int MODE, int PARAM, int PF>
cudaError_t launch_spread_v(const qs_launch& L, const float* x, const float* w, cudaStream_t st)
{
    const int copies = MODE == SPREAD_COPIES ? PARAM : 1;
    const int tw = MODE == SPREAD_THREAD ? (PARAM > L.G ? L.G : PARAM) : 0;
    const size_t smem = ((size_t)copies * (L.G + SPREAD_PAD) + (size_t)tw * 256) * sizeof(int);
    auto kern = spread_filter_kernel<W, FUSED, MODE, PARAM, PF>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<L.P, 256, smem, st>>>(L, x, w);
    return cudaGetLastError();
}

template <int W, bool FUSED, int LW>
cudaError_t launch_moment_v(const qs_launch& L, const float* x, const float* w, cudaStream_t st)
{
    const size_t smem = qs_moment_smem(L.G, W, LW > 0);
    auto kern = spread_moment_kernel<W, FUSED, LW, 4>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<L.P, 512, smem, st>>>(L, x, w);
    return cudaGetLastError();
}

template <int W, bool FUSED>
cudaError_t launch_spread_f(const qs_launch& L, const float* x, const float* w, int variant, cudaStream_t st)
{
    switch (variant) {
        case QS_SPREAD_POINT1: return launch_spread_v<W, FUSED, SPREAD_COPIES, 1, 4>(L, x, w, st);
        case QS_SPREAD_POINT2: return launch_spread_v<W, FUSED, SPREAD_COPIES, 2, 4>(L, x, w, st);
        case QS_SPREAD_POINT4: return launch_spread_v<W, FUSED, SPREAD_COPIES, 4, 4>(L, x, w, st);
        case QS_SPREAD_THREAD32: return launch_spread_v<W, FUSED, SPREAD_THREAD, 32, 4>(L, x, w, st);
        case QS_SPREAD_MOMENT: return launch_moment_v<W, FUSED, 0>(L, x, w, st);
        case QS_SPREAD_MOMENTWIN32: return launch_moment_v<W, FUSED, QS_MOMENT_WIN>(L, x, w, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int W>
cudaError_t launch_spread_w(const qs_launch& L, const float* x, const float* w, bool fused, int variant,
                            cudaStream_t st)
{
    return fused ? launch_spread_f<W, true>(L, x, w, variant, st) : launch_spread_f<W, false>(L, x, w, variant, st);
}

template <int W>
cudaError_t launch_interp_w(const qs_launch& L, const float* y, bool fused, cudaStream_t st)
{
    const int tpt = qs_interp_tpt(fused, L.d, L.G);
    const size_t smem = (size_t)2 * (L.G + ROW_PAD + (fused ? 0 : IT_THREADS * tpt)) * sizeof(float);
    const int64_t mt = L.m_end - L.m_base;
    if (mt <= 0) return cudaSuccess;
    const unsigned gx = (unsigned)((mt + (int64_t)IT_THREADS * tpt - 1) / ((int64_t)IT_THREADS * tpt));
    dim3 grid(gx, (unsigned)L.S);
    // the kernel also holds ~8.5 KB of static shared memory, so the opt-in is
    // needed below 48 KB of dynamic memory too; set it on every launch
#define QS_LAUNCH_INTERP(FU, DM, TP)                                                                       \
    do {                                                                                                   \
        auto k_ = interp_kernel<W, FU, DM, TP>;                                                            \
        cudaError_t e_ = cudaFuncSetAttribute(k_, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e_ != cudaSuccess) return e_;                                                                  \
        k_<<<grid, IT_THREADS, smem, st>>>(L, y);                                                          \
    } while (0)
    if (!fused) QS_LAUNCH_INTERP(false, 1, 8);
    else if (L.d <= 4) QS_LAUNCH_INTERP(true, 4, 2);
    else if (L.d <= 8) QS_LAUNCH_INTERP(true, 8, 2);
    else if (L.d <= 16) QS_LAUNCH_INTERP(true, 16, 1);
    else if (L.d <= 32) QS_LAUNCH_INTERP(true, 32, 1);
    else QS_LAUNCH_INTERP(true, 64, 1);
#undef QS_LAUNCH_INTERP
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_spread_grad_w(const qs_launch& L, const float* x, const float* w, int mode, bool fused,
                                 const float* Dd, float* H2, cudaStream_t st)
{
    if (qs_spread_moments(L.G, W)) {
        const size_t cs = (size_t)L.G + SPREAD_PAD;
        const size_t smem = (cs * (qs_moment_count(W) + 1) + cs + (mode == 2 ? (size_t)L.G : 0)) * sizeof(float);
        auto kern = mode == 2 ? (fused ? spread_grad_moment_kernel<W, 2, true> : spread_grad_moment_kernel<W, 2, false>)
                              : (fused ? spread_grad_moment_kernel<W, 1, true> : spread_grad_moment_kernel<W, 1, false>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<L.P, 512, smem, st>>>(L, x, w, Dd, H2);
        return cudaGetLastError();
    }
    const size_t smem = ((size_t)L.G + SPREAD_PAD + (mode == 2 ? (size_t)L.G : 0)) * sizeof(float);
    auto kern = mode == 2 ? (fused ? spread_grad_kernel<W, 2, true> : spread_grad_kernel<W, 2, false>)
                          : (fused ? spread_grad_kernel<W, 1, true> : spread_grad_kernel<W, 1, false>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<L.P, 256, smem, st>>>(L, x, w, Dd, H2);
    return cudaGetLastError();
}

template <int W, bool FUSED>
void launch_interp_grad_f(const qs_launch& L, const float* y, const float* Hd, const float* xi, float* part,
                          cudaStream_t st)
{
    dim3 grid((unsigned)((L.M + 255) / 256), (unsigned)L.S);
    if (L.d <= 4)
        interp_grad_kernel<W, 4, FUSED><<<grid, 256, 0, st>>>(L, y, Hd, xi, part);
    else if (L.d <= 8)
        interp_grad_kernel<W, 8, FUSED><<<grid, 256, 0, st>>>(L, y, Hd, xi, part);
    else if (L.d <= 16)
        interp_grad_kernel<W, 16, FUSED><<<grid, 256, 0, st>>>(L, y, Hd, xi, part);
    else
        interp_grad_kernel<W, 32, FUSED><<<grid, 256, 0, st>>>(L, y, Hd, xi, part);
}

template <int W>
cudaError_t launch_interp_grad_w(const qs_launch& L, const float* y, const float* Hd, const float* xi, float* part,
                                 bool fused, cudaStream_t st)
{
    if (L.d > QS_GRAD_MAX_D) return cudaErrorInvalidValue;
    if (fused) launch_interp_grad_f<W, true>(L, y, Hd, xi, part, st);
    else launch_interp_grad_f<W, false>(L, y, Hd, xi, part, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t qs_launch_deriv_table(const double* c, const double* psihat, int n_ft, int G, float* Dd, cudaStream_t st)
{
    deriv_table_kernel<<<(G / 2 + 1 + 127) / 128, 128, 0, st>>>(c, psihat, n_ft, G, Dd);
    return cudaGetLastError();
}

cudaError_t qs_launch_spread_grad(const qs_launch& L, int W, const float* x, const float* w, int mode, bool fused,
                                  const float* Dd, float* H2, cudaStream_t st)
{
    switch (W) {
        case 6: return launch_spread_grad_w<6>(L, x, w, mode, fused, Dd, H2, st);
        case 8: return launch_spread_grad_w<8>(L, x, w, mode, fused, Dd, H2, st);
        case 10: return launch_spread_grad_w<10>(L, x, w, mode, fused, Dd, H2, st);
        case 12: return launch_spread_grad_w<12>(L, x, w, mode, fused, Dd, H2, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t qs_launch_interp_grad(const qs_launch& L, int W, const float* y, const float* Hd, const float* xi,
                                  float* part, bool fused, cudaStream_t st)
{
    switch (W) {
        case 6: return launch_interp_grad_w<6>(L, y, Hd, xi, part, fused, st);
        case 8: return launch_interp_grad_w<8>(L, y, Hd, xi, part, fused, st);
        case 10: return launch_interp_grad_w<10>(L, y, Hd, xi, part, fused, st);
        case 12: return launch_interp_grad_w<12>(L, y, Hd, xi, part, fused, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t qs_launch_interp_deriv(const qs_launch& L, int W, const float* Hd, cudaStream_t st)
{
    if (L.M <= 0) return cudaSuccess;
    dim3 grid((unsigned)((L.M + 256 * ID_TPT - 1) / (256 * ID_TPT)), (unsigned)L.P);
    const size_t smem = ((size_t)L.G + ROW_PAD) * sizeof(float);
#define QS_LAUNCH_DERIV(WW)                                                                                 \
    do {                                                                                                    \
        cudaError_t e_ = cudaFuncSetAttribute(interp_deriv_kernel<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)smem);                                                   \
        if (e_ != cudaSuccess) return e_;                                                                   \
        interp_deriv_kernel<WW><<<grid, 256, smem, st>>>(L, Hd);                                            \
    } while (0)
    switch (W) {
        case 6: QS_LAUNCH_DERIV(6); break;
        case 8: QS_LAUNCH_DERIV(8); break;
        case 10: QS_LAUNCH_DERIV(10); break;
        case 12: QS_LAUNCH_DERIV(12); break;
        default: return cudaErrorInvalidValue;
    }
#undef QS_LAUNCH_DERIV
    return cudaGetLastError();
}

cudaError_t qs_launch_backproj(const float* Q, int64_t ldQ, int64_t M, int P, const float* xi, int d, float scale,
                               const float* fac, float* out, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    // tiles (targets x components): 256 x 16 and 128 x 32 (4 x 4 outputs per thread), 128 x 64 (8 x 4)
    if (d <= 16) {
        dim3 grid((unsigned)((M + 255) / 256), (unsigned)((d + 15) / 16));
        backproj_kernel<16, 4><<<grid, 256, 0, st>>>(Q, ldQ, M, P, xi, d, scale, fac, out);
    } else if (d <= 32) {
        dim3 grid((unsigned)((M + 127) / 128), (unsigned)((d + 31) / 32));
        backproj_kernel<32, 4><<<grid, 256, 0, st>>>(Q, ldQ, M, P, xi, d, scale, fac, out);
    } else {
        dim3 grid((unsigned)((M + 127) / 128), (unsigned)((d + 63) / 64));
        backproj_kernel<64, 8><<<grid, 256, 0, st>>>(Q, ldQ, M, P, xi, d, scale, fac, out);
    }
    return cudaGetLastError();
}

cudaError_t qs_launch_reduce_grad(const float* part, int S, int64_t M, int d, float scale, const float* fac,
                                  float* out, cudaStream_t st)
{
    const int64_t n = M * d;
    reduce_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, S, M, d, scale, fac, out);
    return cudaGetLastError();
}

cudaError_t qs_launch_coeffs(int kernel, double kparam, double kparam2, int d, double tau, int n_ft, int G,
                             const double* psihat, const double* c_in, double* c_out, float* D_out, cudaStream_t st)
{
    const int n = (n_ft > G / 2 + 1 ? n_ft : G / 2 + 1);
    coeff_kernel<<<(n + 127) / 128, 128, 0, st>>>(kernel, kparam, kparam2, d, tau, n_ft, G, psihat, c_in, c_out,
                                                   D_out);
    return cudaGetLastError();
}

cudaError_t qs_launch_weight_scale(const qs_launch& L, const float* w, cudaStream_t st)
{
    weight_scale_kernel<<<1, 1024, 0, st>>>(w, L.N, L.wscale, L.flag);
    return cudaGetLastError();
}

cudaError_t qs_launch_spread(const qs_launch& L, int W, const float* x, const float* w, bool fused,
                             cudaStream_t st)
{
    if (!qs_spread_variant_ok(L.G, W, L.spread_variant)) return cudaErrorInvalidValue;
    switch (W) {
        case 6: return launch_spread_w<6>(L, x, w, fused, L.spread_variant, st);
        case 8: return launch_spread_w<8>(L, x, w, fused, L.spread_variant, st);
        case 10: return launch_spread_w<10>(L, x, w, fused, L.spread_variant, st);
        case 12: return launch_spread_w<12>(L, x, w, fused, L.spread_variant, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t qs_launch_interp(const qs_launch& L, int W, const float* y, bool fused, cudaStream_t st)
{
    switch (W) {
        case 6: return launch_interp_w<6>(L, y, fused, st);
        case 8: return launch_interp_w<8>(L, y, fused, st);
        case 10: return launch_interp_w<10>(L, y, fused, st);
        case 12: return launch_interp_w<12>(L, y, fused, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t qs_launch_reduce(const qs_launch& L, float* s, cudaStream_t st)
{
    reduce_kernel<<<(unsigned)((L.M + 255) / 256), 256, 0, st>>>(L.part, L.S, L.M, L.P, s);
    return cudaGetLastError();
}
