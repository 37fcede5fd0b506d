// Sorting slicing for the negative distance kernel F(r) = -r (Sec. 2.1,
// eq. kernel_sum_sliced, with the one-dimensional basis function
// f(t) = -c_d |t| of Table tab:kernels; the sorting evaluation of the 1D sums
// that the paper uses for this kernel in its MMD-flow experiments):
//
//   s_m = (1/P) sum_p sum_n w_n f(|<x_n - y_m, xi_p>|)
//
// exactly, without Fourier truncation.  Per slice, with a_n, b_m the
// projections, sort sources and targets together; with W_<(b) and S_<(b) the
// sums of w_n and w_n a_n over the sources before b in that order,
//   sum_n w_n |b - a_n| = b (2 W_< - W) - (2 S_< - S),    W, S the totals,
// one FP64 scan per slice.  (Sources equal to b contribute 0 on either side.)
//
// Slices are processed in chunks of CS.  Per chunk: an init kernel forms the
// FP32 projections (the dot products of the fused form) as order-preserving
// 32-bit keys with the point index as payload; four stable LSD radix passes
// of 8 bits (per-tile digit histograms, a per-slice scan, a scatter that
// ranks within each warp with __match_any_sync); FP64 sums per sorted tile, a
// per-slice scan of those, and a per-tile evaluation that adds the tile's
// prefix; then a TwoSum accumulation of the chunk's slice values in slice
// order.  Every sum has a fixed order, so results are reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qs_internal.cuh"

namespace {

constexpr int SORT_TILE = 2048;      // elements per tile of a radix pass
constexpr int SORT_THREADS = 256;
constexpr int SORT_ROUNDS = SORT_TILE / SORT_THREADS;

__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// keys[pl][i]: projection of source i (i < N) or target i - N on slice p0 + pl,
// u = <xi_s_p, point> in the grid units of the plan (FP32, j order).
__global__ void sort_init_kernel(const float* __restrict__ x, int64_t N, const float* __restrict__ y, int64_t M,
                                 const float* __restrict__ xi_s, int d, int p0, int64_t LS,
                                 uint32_t* __restrict__ key, uint32_t* __restrict__ pay, unsigned int* flag)
{
    __shared__ float xs[QS_FUSED_MAX_D];
    const int pl = blockIdx.y;
    for (int j = threadIdx.x; j < d; j += blockDim.x) xs[j] = xi_s[(size_t)(p0 + pl) * d + j];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N + M) return;
    const float* pt = i < N ? x + (size_t)i * d : y + (size_t)(i - N) * d;
    float u = 0.0f;
    for (int j = 0; j < d; ++j) u = fmaf(xs[j], __ldg(&pt[j]), u);
    if (!isfinite(u)) {
        atomicOr(flag, QS_FLAG_NONFINITE);
        u = 0.0f;
    }
    key[(size_t)pl * LS + i] = float_key(u);
    pay[(size_t)pl * LS + i] = (uint32_t)i;
}

// hist[(pl * 256 + digit) * T + tile] = count of the digit in the tile
__global__ void __launch_bounds__(SORT_THREADS) sort_hist_kernel(const uint32_t* __restrict__ key, int64_t L,
                                                                 int64_t LS, int T, int shift,
                                                                 uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[256];
    const int t = blockIdx.x, pl = blockIdx.y;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t* k = key + (size_t)pl * LS;
    const int64_t e0 = (int64_t)t * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t e = e0 + r * SORT_THREADS + threadIdx.x;
        if (e < L) atomicAdd(&h[(k[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[((size_t)pl * 256 + threadIdx.x) * T + t] = h[threadIdx.x];
}

// per slice: exclusive scan of its 256 x T counts (digit-major), in place
__global__ void __launch_bounds__(1024) sort_scan_kernel(uint32_t* __restrict__ hist, int T)
{
    __shared__ uint32_t part[1024];
    uint32_t* h = hist + (size_t)blockIdx.x * 256 * T;
    const int n = 256 * T;
    const int per = (n + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(n, b + per);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += h[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = b; i < e; ++i) {
        const uint32_t c = h[i];
        h[i] = run;
        run += c;
    }
}

// stable scatter of one tile: element order (round, thread) is index order
__global__ void __launch_bounds__(SORT_THREADS) sort_scatter_kernel(const uint32_t* __restrict__ kin,
                                                                    const uint32_t* __restrict__ pin, int64_t L,
                                                                    int64_t LS, int T, int shift,
                                                                    const uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ kout,
                                                                    uint32_t* __restrict__ pout)
{
    __shared__ uint32_t gbase[256], base[256];
    __shared__ uint32_t wc[2][SORT_THREADS / 32][256];
    const int t = blockIdx.x, pl = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    gbase[threadIdx.x] = hist[((size_t)pl * 256 + threadIdx.x) * T + t];
    base[threadIdx.x] = 0;
    for (int w = 0; w < SORT_THREADS / 32; ++w) {
        wc[0][w][threadIdx.x] = 0;
        wc[1][w][threadIdx.x] = 0;
    }
    __syncthreads();
    const uint32_t* ki = kin + (size_t)pl * LS;
    const uint32_t* pi = pin + (size_t)pl * LS;
    uint32_t* ko = kout + (size_t)pl * LS;
    uint32_t* po = pout + (size_t)pl * LS;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t e0 = (int64_t)t * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int b = r & 1;
        const int64_t e = e0 + r * SORT_THREADS + threadIdx.x;
        const bool active = e < L;
        const uint32_t k = active ? ki[e] : 0u;
        const uint32_t pv = active ? pi[e] : 0u;
        const uint32_t dg = active ? ((k >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt);
        if (active && rank == 0) wc[b][warp][dg] = __popc(peers);
        __syncthreads();
        {
            // digit threadIdx.x: exclusive offsets of the warps, after the earlier rounds;
            // the other buffer is cleared for the next round
            uint32_t run = base[threadIdx.x];
            for (int w = 0; w < SORT_THREADS / 32; ++w) {
                const uint32_t c = wc[b][w][threadIdx.x];
                wc[b][w][threadIdx.x] = run;
                run += c;
                wc[b ^ 1][w][threadIdx.x] = 0;
            }
            base[threadIdx.x] = run;
        }
        __syncthreads();
        if (active) {
            const uint32_t pos = gbase[dg] + wc[b][warp][dg] + rank;
            ko[pos] = k;
            po[pos] = pv;
        }
    }
}

// FP64 sums of (w, w a) over the sources of each sorted tile (fixed order)
__global__ void __launch_bounds__(SORT_THREADS) sort_tilesum_kernel(const uint32_t* __restrict__ key,
                                                                    const uint32_t* __restrict__ pay, int64_t N,
                                                                    int64_t L, int64_t LS, int T,
                                                                    const float* __restrict__ w,
                                                                    double* __restrict__ tsum)
{
    __shared__ double rw[SORT_THREADS / 32], ra[SORT_THREADS / 32];
    const int t = blockIdx.x, pl = blockIdx.y;
    const uint32_t* k = key + (size_t)pl * LS;
    const uint32_t* p = pay + (size_t)pl * LS;
    double sw = 0.0, sa = 0.0;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t e = (int64_t)t * SORT_TILE + r * SORT_THREADS + threadIdx.x;
        if (e < L) {
            const uint32_t i = p[e];
            if (i < N) {
                const double wn = w ? (double)w[i] : 1.0;
                sw += wn;
                sa += wn * (double)key_float(k[e]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rw[threadIdx.x >> 5] = sw;
        ra[threadIdx.x >> 5] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0, ta = 0.0;
        for (int q = 0; q < SORT_THREADS / 32; ++q) {
            tw += rw[q];
            ta += ra[q];
        }
        tsum[((size_t)pl * T + t) * 2 + 0] = tw;
        tsum[((size_t)pl * T + t) * 2 + 1] = ta;
    }
}

// per slice, serially: exclusive prefix of the tile sums in place, totals in tot[pl]
__global__ void sort_tilescan_kernel(double* __restrict__ tsum, int T, int cs, double* __restrict__ tot)
{
    const int pl = blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= cs) return;
    double* ts = tsum + (size_t)pl * T * 2;
    double rw = 0.0, ra = 0.0;
    for (int t = 0; t < T; ++t) {
        const double cw = ts[2 * t], ca = ts[2 * t + 1];
        ts[2 * t] = rw;
        ts[2 * t + 1] = ra;
        rw += cw;
        ra += ca;
    }
    tot[2 * pl] = rw;
    tot[2 * pl + 1] = ra;
}

// per sorted tile: exclusive FP64 prefix of (w, w a) over the sources before
// each element; for every target m the slice's value
// amp * (b (2 W_< - W) - (2 S_< - S)) goes to t[pl][m]
// GRAD: t[pl][m] = 2 W_< - W = sum_n w_n sign(b - a_n) instead (sources whose
// key equals b's sort before it and count as below: a one-sided subgradient)
template <bool GRAD>
__global__ void __launch_bounds__(SORT_THREADS) sort_eval_kernel(const uint32_t* __restrict__ key,
                                                                 const uint32_t* __restrict__ pay, int64_t N,
                                                                 int64_t M, int64_t LS, int T,
                                                                 const float* __restrict__ w,
                                                                 const double* __restrict__ tsum,
                                                                 const double* __restrict__ tot, double amp,
                                                                 float* __restrict__ tout)
{
    __shared__ double sw[SORT_THREADS / 32], sa[SORT_THREADS / 32];
    const int t = blockIdx.x, pl = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t* k = key + (size_t)pl * LS;
    const uint32_t* p = pay + (size_t)pl * LS;
    const int64_t L = N + M;
    const double W = tot[2 * pl], S = tot[2 * pl + 1];
    double carry_w = tsum[((size_t)pl * T + t) * 2 + 0];
    double carry_a = tsum[((size_t)pl * T + t) * 2 + 1];
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t e = (int64_t)t * SORT_TILE + r * SORT_THREADS + threadIdx.x;
        double vw = 0.0, va = 0.0, b = 0.0;
        uint32_t i = 0xffffffffu;
        if (e < L) {
            i = p[e];
            b = (double)key_float(k[e]);
            if (i < N) {
                vw = w ? (double)w[i] : 1.0;
                va = vw * b;
            }
        }
        double iw = vw, ia = va;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const double nw = __shfl_up_sync(0xffffffffu, iw, o);
            const double na = __shfl_up_sync(0xffffffffu, ia, o);
            if (lane >= o) {
                iw += nw;
                ia += na;
            }
        }
        if (lane == 31) {
            sw[warp] = iw;
            sa[warp] = ia;
        }
        __syncthreads();
        double ow = carry_w, oa = carry_a, bw = carry_w, ba = carry_a;
        for (int q = 0; q < SORT_THREADS / 32; ++q) {
            if (q < warp) {
                ow += sw[q];
                oa += sa[q];
            }
            bw += sw[q];
            ba += sa[q];
        }
        if (e < L && i >= N) {
            const double Wl = ow + iw - vw, Sl = oa + ia - va;  // sources strictly before
            tout[(size_t)pl * M + (i - N)] =
                GRAD ? (float)(2.0 * Wl - W) : (float)(amp * (b * (2.0 * Wl - W) - (2.0 * Sl - S)));
        }
        carry_w = bw;
        carry_a = ba;
        __syncthreads();
    }
}

// hi/lo += t[pl][m] for pl = 0 .. CS-1 in order (TwoSum)
__global__ void sort_accum_kernel(const float* __restrict__ t, int CS, int64_t M, float* __restrict__ hi,
                                  float* __restrict__ lo)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float h = hi[m], l = lo[m];
    for (int pl = 0; pl < CS; ++pl) qs_two_sum(h, l, t[(size_t)pl * M + m]);
    hi[m] = h;
    lo[m] = l;
}

// gradient accumulators ghi/glo [j][m] += t[pl][m] xi_{p0+pl}[j], pl in order (TwoSum)
__global__ void sort_gaccum_kernel(const float* __restrict__ t, int CS, int64_t M, const float* __restrict__ xi,
                                   int d, int p0, float* __restrict__ ghi, float* __restrict__ glo)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int j = 0; j < d; ++j) {
        float h = ghi[(size_t)j * M + m], l = glo[(size_t)j * M + m];
        for (int pl = 0; pl < CS; ++pl) qs_two_sum(h, l, t[(size_t)pl * M + m] * __ldg(&xi[(size_t)(p0 + pl) * d + j]));
        ghi[(size_t)j * M + m] = h;
        glo[(size_t)j * M + m] = l;
    }
}

// gy[m][j] = v_m scale (hi + lo)
__global__ void sort_gfinal_kernel(const float* __restrict__ ghi, const float* __restrict__ glo, int64_t M, int d,
                                   const float* __restrict__ v, float scale, float* __restrict__ gy)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const float vm = (v ? v[m] : 1.0f) * scale;
    for (int j = 0; j < d; ++j) gy[(size_t)m * d + j] = vm * (ghi[(size_t)j * M + m] + glo[(size_t)j * M + m]);
}

__global__ void sort_final_kernel(const float* __restrict__ hi, const float* __restrict__ lo, int64_t M, int P,
                                  float* __restrict__ s)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) s[m] = (hi[m] + lo[m]) / (float)P;
}

}  // namespace

// Chunk of slices and the workspace for up to L = N + M points.
int qs_sort_chunk(int P) { return P < 32 ? P : 32; }

size_t qs_sort_workspace_bytes(int P, int64_t max_n, int64_t max_m)
{
    const int CS = qs_sort_chunk(P);
    const int64_t L = max_n + max_m;
    const int64_t LS = (L + SORT_TILE - 1) / SORT_TILE * SORT_TILE;
    const int64_t T = LS / SORT_TILE;
    return (size_t)4 * CS * LS * sizeof(uint32_t)         // key / payload, two buffers each
           + (size_t)CS * 256 * T * sizeof(uint32_t)      // digit offsets
           + (size_t)CS * T * 2 * sizeof(double)          // tile sums
           + (size_t)CS * 2 * sizeof(double)              // slice totals
           + (size_t)CS * max_m * sizeof(float)           // slice values of a chunk
           + (size_t)2 * max_m * QS_FUSED_MAX_D * sizeof(float) + 1024;  // hi / lo (x d for gradients)
}

// s != NULL: the sum; else gy (M x d) = v_m (-c_d/P) sum_p (sum_n w_n sign(b - a_n)) xi_p,
// with `scale` = -c_d / P and xi the unscaled directions.
cudaError_t qs_launch_sum_sorted(const float* x, int64_t N, const float* w, const float* y, int64_t M,
                                 const float* xi_s, const float* xi, int d, int P, double amp, void* ws,
                                 int64_t max_n, int64_t max_m, float* s, const float* v, float scale, float* gy,
                                 unsigned int* flag, cudaStream_t st)
{
    const bool grad = s == nullptr;
    if (M <= 0) return cudaSuccess;
    const int CS = qs_sort_chunk(P);
    const int64_t L = N + M;
    const int64_t Lmax = max_n + max_m;
    const int64_t LS = (Lmax + SORT_TILE - 1) / SORT_TILE * SORT_TILE;
    const int Tmax = (int)(LS / SORT_TILE);
    const int T = (int)((L + SORT_TILE - 1) / SORT_TILE);
    uint8_t* b = reinterpret_cast<uint8_t*>(ws);
    uint32_t* kA = reinterpret_cast<uint32_t*>(b);
    uint32_t* pA = kA + (size_t)CS * LS;
    uint32_t* kB = pA + (size_t)CS * LS;
    uint32_t* pB = kB + (size_t)CS * LS;
    uint32_t* hist = pB + (size_t)CS * LS;
    double* tsum = reinterpret_cast<double*>(hist + (size_t)CS * 256 * Tmax);  // 8-byte aligned: even count
    double* tot = tsum + (size_t)CS * Tmax * 2;
    float* tb = reinterpret_cast<float*>(tot + (size_t)CS * 2);
    float* hi = tb + (size_t)CS * max_m;
    float* lo = hi + max_m;
    const size_t acc = (size_t)M * (grad ? d : 1);  // accumulators of this call, hi then lo
    lo = hi + acc;
    cudaError_t e = cudaMemsetAsync(hi, 0, sizeof(float) * 2 * acc, st);
    for (int p0 = 0; p0 < P && e == cudaSuccess; p0 += CS) {
        const int cs = P - p0 < CS ? P - p0 : CS;
        sort_init_kernel<<<dim3((unsigned)((L + 255) / 256), (unsigned)cs), 256, 0, st>>>(x, N, y, M, xi_s, d, p0, LS,
                                                                                          kA, pA, flag);
        uint32_t *ki = kA, *pi = pA, *ko = kB, *po = pB;
        for (int shift = 0; shift < 32 && (e = cudaGetLastError()) == cudaSuccess; shift += 8) {
            sort_hist_kernel<<<dim3((unsigned)T, (unsigned)cs), SORT_THREADS, 0, st>>>(ki, L, LS, T, shift, hist);
            sort_scan_kernel<<<cs, 1024, 0, st>>>(hist, T);
            sort_scatter_kernel<<<dim3((unsigned)T, (unsigned)cs), SORT_THREADS, 0, st>>>(ki, pi, L, LS, T, shift,
                                                                                         hist, ko, po);
            uint32_t* tk = ki;
            ki = ko;
            ko = tk;
            tk = pi;
            pi = po;
            po = tk;
        }
        if (e != cudaSuccess) break;
        // four passes: the sorted data are back in the A buffers
        sort_tilesum_kernel<<<dim3((unsigned)T, (unsigned)cs), SORT_THREADS, 0, st>>>(ki, pi, N, L, LS, T, w, tsum);
        sort_tilescan_kernel<<<1, 32, 0, st>>>(tsum, T, cs, tot);
        const dim3 eg((unsigned)T, (unsigned)cs);
        if (grad) {
            sort_eval_kernel<true><<<eg, SORT_THREADS, 0, st>>>(ki, pi, N, M, LS, T, w, tsum, tot, amp, tb);
            sort_gaccum_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(tb, cs, M, xi, d, p0, hi, lo);
        } else {
            sort_eval_kernel<false><<<eg, SORT_THREADS, 0, st>>>(ki, pi, N, M, LS, T, w, tsum, tot, amp, tb);
            sort_accum_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(tb, cs, M, hi, lo);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (grad)
            sort_gfinal_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(hi, lo, M, d, v, scale, gy);
        else
            sort_final_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(hi, lo, M, P, s);
        e = cudaGetLastError();
    }
    return e;
}
