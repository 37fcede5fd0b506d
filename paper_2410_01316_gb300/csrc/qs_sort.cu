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
// one prefix scan per slice.  (Sources equal to b contribute 0 on either side.)
//
// Slices are processed in chunks of CS.  Per chunk: the FP32 SIMT GEMM forms
// the chunk's projections of sources and targets (one fmaf chain per pair in
// j order); four stable LSD radix passes of 8 bits sort them as
// order-preserving 32-bit keys with the point index as payload (the first
// pass reads the projections directly), each pass a per-tile digit
// histogram, a per-slice scan and a scatter that ranks within each warp by
// ballots on the digit's bits, stages the tile in digit order in shared
// memory and writes each digit's run with consecutive threads; then 64-bit
// fixed-point sums of w and w a per sorted tile, a per-slice scan of those,
// and a per-tile evaluation that adds the tile's prefix (integer sums are
// exact, so their order does not matter; the per-target formula in
// error-free FP32 arithmetic); then a TwoSum accumulation of the chunk's
// slice values in slice order, and the kernel's factor once per target.
// Results are reproducible.
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

// Where a radix pass reads element e of slice pl: the previous pass's keys
// and payloads, or (first pass) the chunk's projections proj[pl][.] (sources
// at columns 0 .. N-1, targets from column Nr = N rounded up to 128), which
// the FP32 SIMT GEMM formed as one fmaf chain in j order per (slice, point),
// turned into order-preserving keys with the point index as payload.  A
// non-finite projection sorts as 0 and raises the data flag (in the first
// histogram pass).
struct KeySrc {
    const uint32_t* key;
    const uint32_t* pay;
    const float* proj;
    int64_t N, Nr, ldp;
    unsigned int* flag;
};

template <bool FROM_PROJ>
__device__ __forceinline__ uint32_t src_key(const KeySrc& s, int pl, int64_t LS, int64_t e, bool check)
{
    if (FROM_PROJ) {
        float u = __ldg(&s.proj[(size_t)pl * s.ldp + (e < s.N ? e : s.Nr + (e - s.N))]);
        if (!isfinite(u)) {
            if (check) atomicOr(s.flag, QS_FLAG_NONFINITE);
            u = 0.0f;
        }
        return float_key(u);
    }
    return __ldg(&s.key[(size_t)pl * LS + e]);
}

template <bool FROM_PROJ>
__device__ __forceinline__ uint32_t src_pay(const KeySrc& s, int pl, int64_t LS, int64_t e)
{
    return FROM_PROJ ? (uint32_t)e : __ldg(&s.pay[(size_t)pl * LS + e]);
}

// The lanes of the warp whose 8-bit digit equals this lane's: the AND over the
// digit's bits of the ballot of that bit (or of its complement), restricted to
// the active lanes (dg < 256); an inactive lane (dg = 256) gets 0.  Eight
// ballots cost less than __match_any_sync, which throttles the MIO pipe here.
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg)
{
    uint32_t peers = __ballot_sync(0xffffffffu, dg < 256u);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (dg >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return dg < 256u ? peers : 0u;
}

// hist[(pl * 256 + digit) * T + tile] = count of the digit in the tile, by
// shared-memory atomics (three of the four digits of a projection's key are
// close to uniform, so lanes rarely collide; aggregating equal digits first
// costs more issue slots than the collisions of the top digit)
template <bool FROM_PROJ>
__global__ void __launch_bounds__(SORT_THREADS) sort_hist_kernel(KeySrc src, int64_t L, int64_t LS, int T,
                                                                 int shift, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[256];
    const int t = blockIdx.x, pl = blockIdx.y;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t e0 = (int64_t)t * SORT_TILE;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t e = e0 + r * SORT_THREADS + threadIdx.x;
        if (e < L) atomicAdd(&h[(src_key<FROM_PROJ>(src, pl, LS, e, true) >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[((size_t)pl * 256 + threadIdx.x) * T + t] = h[threadIdx.x];
}

// per slice: exclusive scan of its 256 x T counts (digit-major), in place,
// 4096 entries at a time (four consecutive per thread, 16-byte accesses; the
// count array of a slice starts on a 16-byte boundary because 256 T is a
// multiple of 4): a block scan of the threads' sums plus the running carry
__global__ void __launch_bounds__(1024) sort_scan_kernel(uint32_t* __restrict__ hist, int T)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry_s;
    uint4* h4 = reinterpret_cast<uint4*>(hist + (size_t)blockIdx.x * 256 * T);
    const int n4 = 64 * T;  // 256 T / 4
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < n4; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        uint4 v = i < n4 ? h4[i] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t tsum = v.x + v.y + v.z + v.w;
        uint32_t inc = tsum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t nv = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += nv;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t x = wsum[lane];
            uint32_t y = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nv = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += nv;
            }
            wsum[lane] = y - x;  // exclusive over the warps
            if (lane == 31) carry_s = y;
        }
        __syncthreads();
        uint32_t run = carry + wsum[warp] + inc - tsum;
        const uint32_t block_total = carry_s;
        if (i < n4) {
            uint4 o;
            o.x = run;
            run += v.x;
            o.y = run;
            run += v.y;
            o.z = run;
            run += v.z;
            o.w = run;
            h4[i] = o;
        }
        carry += block_total;
        __syncthreads();  // wsum and carry_s are rewritten by the next block of entries
    }
}

// Stable scatter of one tile.  Warp w ranks the w-th run of SORT_TILE / NW
// consecutive elements, 32 at a time, against its own digit counters (lanes
// with equal digits found by digit_peers; the first of them updates the
// counter), so no block barrier is needed until the tile is ranked; then one
// pass over the 256 digits turns the warps' counts into offsets, the tile is
// placed in digit order in shared memory, and written out with consecutive
// threads on consecutive positions of each digit's run.  The tile's count of
// a digit is the difference of consecutive scanned offsets in the flattened
// (digit, tile) order.
template <bool FROM_PROJ>
__global__ void __launch_bounds__(SORT_THREADS, 6) sort_scatter_kernel(KeySrc src, int64_t L, int64_t LS, int T,
                                                                    int shift, const uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ kout,
                                                                    uint32_t* __restrict__ pout)
{
    constexpr int NW = SORT_THREADS / 32;
    constexpr int R = SORT_TILE / SORT_THREADS;  // rounds of 32 elements per warp
    __shared__ uint32_t gbase[256], lbase[256], wsum[NW];
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t sk[SORT_TILE], sp[SORT_TILE];
    const int t = blockIdx.x, pl = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const size_t flat = ((size_t)pl * 256 + threadIdx.x) * T + t;
        const uint32_t g0 = hist[flat];
        const uint32_t g1 = (threadIdx.x == 255 && t == T - 1) ? (uint32_t)L : hist[flat + 1];
        gbase[threadIdx.x] = g0;
        // exclusive scan of the tile's digit counts over the 256 digits
        const uint32_t c = g1 - g0;
        uint32_t inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        if (lane == 31) wsum[warp] = inc;
        for (int w = 0; w < NW; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        uint32_t off = 0;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        lbase[threadIdx.x] = off + inc - c;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t e0 = (int64_t)t * SORT_TILE + (int64_t)warp * (R * 32);
    uint32_t kk[R], pp[R], rk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {  // all loads first: 2 R in flight per thread
        const int64_t e = e0 + r * 32 + lane;
        kk[r] = e < L ? src_key<FROM_PROJ>(src, pl, LS, e, false) : 0u;
        pp[r] = e < L ? src_pay<FROM_PROJ>(src, pl, LS, e) : 0u;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool active = e0 + r * 32 + lane < L;
        const uint32_t dg = active ? ((kk[r] >> shift) & 255u) : 256u;
        const uint32_t peers = digit_peers(dg);
        const int leader = peers ? __ffs(peers) - 1 : 0;
        uint32_t before = 0;
        if (active && lane == leader) {
            before = wcnt[warp][dg];
            wcnt[warp][dg] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rk[r] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        // digit threadIdx.x: exclusive offsets of the warps' runs, in warp order
        uint32_t run = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (e0 + r * 32 + lane < L) {
            const uint32_t dg = (kk[r] >> shift) & 255u;
            const uint32_t lp = lbase[dg] + wcnt[warp][dg] + rk[r];
            sk[lp] = kk[r];
            sp[lp] = pp[r];
        }
    }
    __syncthreads();
    uint32_t* ko = kout + (size_t)pl * LS;
    uint32_t* po = pout + (size_t)pl * LS;
    const int n = (int)min((int64_t)SORT_TILE, L - (int64_t)t * SORT_TILE);
    for (int j = threadIdx.x; j < n; j += SORT_THREADS) {
        const uint32_t k = sk[j];
        const uint32_t dg = (k >> shift) & 255u;
        const uint32_t pos = gbase[dg] + (uint32_t)j - lbase[dg];
        ko[pos] = k;
        po[pos] = sp[j];
    }
}

// The prefix sums W_< = sum of w_n and S_< = sum of w_n a_n over the sources
// before a target run in 64-bit fixed point: each source contributes
// qw = [w 2^ew] and qs = [w a 2^es], [.] rounding to nearest (w a is the
// exact integer product of the two significands, rounded once), with powers of
// two chosen per slice so that every partial sum stays below 2^51 in
// magnitude: sum|w| <= N max|w| and max|a| <= the larger of the slice's first
// and last sorted keys in magnitude.  Integer sums are exact and do not depend
// on their order.  Everything per element is integer or FP32 arithmetic (FP64
// is slow on this GPU): a target's value comes from the prefix sums by
// splitting them into two exact FP32 parts and combining them with
// error-free products and sums.
struct SortScale {
    unsigned int wmax;    // bits of max |w| over the sources (a float >= 0; order-independent)
};

struct SliceScale {
    int ew, es;           // fixed-point exponents of w and w a
    float c1, c2;         // 2^(es - ew) as two factors (the units of 2^-ew into those of 2^-es)
    float s1, s2;         // 2^-es as two factors
    float g1, g2;         // 2^-ew as two factors
};

// 2^k as a float, -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// 2^k as two normal-float factors, |k| <= 252
__device__ __forceinline__ void pow2_pair(int k, float& f1, float& f2)
{
    const int k1 = k / 2;
    f1 = pow2f(k1);
    f2 = pow2f(k - k1);
}

// k with |x| < 2^k for a finite float x (from its exponent field; denormals and 0 give -126)
__device__ __forceinline__ int pow2_above(float x) { return (int)((__float_as_uint(x) >> 23) & 255u) - 126; }

// The scales of one slice from max|w| and the slice's sorted keys k[0 .. L-1]:
// N <= 2^lgN, so sum |w| < 2^(lgN + pow2_above(max|w|)) and sum |w a| below that times
// 2^pow2_above(max|a|); ew, es leave sum |qw| < 2^51 + N / 2 and sum |qs| < 2^50 + N / 2.
__device__ __forceinline__ SliceScale slice_scale(const SortScale* rec, bool unit_w, int64_t N,
                                                  const uint32_t* k, int64_t L)
{
    const float wm = unit_w ? 1.0f : __uint_as_float(rec->wmax);
    const float am = fmaxf(fabsf(key_float(k[0])), fabsf(key_float(k[L - 1])));
    const int lgN = N > 1 ? 64 - __clzll((unsigned long long)(N - 1)) : 0;
    SliceScale sc;
    sc.ew = 51 - (lgN + pow2_above(wm));
    sc.es = 50 - (lgN + pow2_above(wm) + pow2_above(am));
    if (sc.es > 250) sc.es = 250;  // only for max|w| max|a| below ~1e-61: a coarser unit, the same bound
    pow2_pair(sc.es - sc.ew, sc.c1, sc.c2);
    pow2_pair(-sc.es, sc.s1, sc.s2);
    pow2_pair(-sc.ew, sc.g1, sc.g2);
    return sc;
}

// max |w| over the sources as the bits of a non-negative float (atomicMax on
// the bits is order-independent); non-finite weights raise the data flag.
// rec->wmax is cleared before the launch.
__global__ void sort_wmax_kernel(const float* __restrict__ w, int64_t N, SortScale* __restrict__ rec,
                                 unsigned int* flag)
{
    unsigned int m = 0u;
    bool bad = false;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float a = fabsf(w[n]);
        if (a <= 3.4e38f) m = max(m, __float_as_uint(a));
        else bad = true;
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&rec->wmax, m);
    if (bad) atomicOr(flag, QS_FLAG_NONFINITE);
}

// A finite float as (-1)^neg m 2^(e - 150) with 2^23 <= m < 2^24 for every
// nonzero x (denormals normalised), m = 0 for zeros
struct FDec {
    uint32_t m;
    int e;
    uint32_t neg;
};

__device__ __forceinline__ FDec fdec(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 255u;
    FDec r;
    const uint32_t m = (b & 0x7fffffu) | (ex ? 0x800000u : 0u);
    const int z = __clz(m) - 8;  // 0 for normal x
    r.m = m << z;
    r.e = (ex ? (int)ex : 1) - z;
    r.neg = b >> 31;
    return r;
}

// (-1)^neg round(t 2^-k), halves away from zero, for t < 2^62 and k clamped to [1, 63]
// (branch-free; with normalised significands the scales keep k >= 4)
__device__ __forceinline__ long long shr_round(unsigned long long t, int k, uint32_t neg)
{
    k = min(max(k, 1), 63);
    const long long v = (long long)((t + (1ull << (k - 1))) >> k);
    return neg ? -v : v;
}

// qw = [w 2^ew] from m_w 2^32 shifted down; qs = [w a 2^es] from the 48-bit
// product m_w m_a, shifted up by 8 and down again (m_w m_a >= 2^46 for nonzero
// inputs and |w a 2^es| < 2^51 keep the shift >= 4; |w 2^ew| < 2^51 keeps the
// shift of qw >= 5)
__device__ __forceinline__ void src_fixed(float wn, float a, const SliceScale& sc, long long& qw, long long& qs)
{
    const FDec dw = fdec(wn), da = fdec(a);
    qw = shr_round((unsigned long long)dw.m << 32, 32 - (dw.e - 150 + sc.ew), dw.neg);
    qs = shr_round(((unsigned long long)dw.m * da.m) << 8, 8 - (dw.e + da.e - 300 + sc.es), dw.neg ^ da.neg);
}

// X (|X| < 2^53) as hi + lo: hi = 2^32 (X >> 32) exactly, lo = fl(X mod 2^32), |lo - (X mod 2^32)| <= 2^7
__device__ __forceinline__ void split_fixed(long long X, float& hi, float& lo)
{
    hi = (float)(int)(X >> 32) * 4294967296.0f;
    lo = (float)(unsigned int)(X & 0xffffffffll);
}

// sum_n w_n |b - a_n| = b (2 W_< - W) - (2 S_< - S) with XW = 2^ew (2 W_< - W),
// XS = 2^es (2 S_< - S), evaluated in the units of 2^-es with an error-free
// product of b and XW's high part and an error-free sum against XS's high part;
// the rest (products' rounding, low parts) is below 2^-40 of the terms.
// |b 2^(es - ew)| <= 1/2: 2^es max|a| and 2^ew differ by at least 2 max|a|.
__device__ __forceinline__ float sorted_value(float b, long long XW, long long XS, const SliceScale& sc)
{
    float wh, wl, sh, sl;
    split_fixed(XW, wh, wl);
    split_fixed(XS, sh, sl);
    wh = wh * sc.c1 * sc.c2;
    wl = wl * sc.c1 * sc.c2;
    const float p1 = b * wh;
    const float e1 = fmaf(b, wh, -p1);
    const float t = p1 - sh;  // TwoSum(p1, -sh)
    const float bv = t - p1;
    const float u = (p1 - (t - bv)) + (-sh - bv);
    const float rest = e1 + fmaf(b, wl, -sl) + u;
    return (t + rest) * sc.s1 * sc.s2;
}

// consecutive elements of a tile per thread, loaded as 16-byte vectors
constexpr int SORT_VPT = SORT_TILE / SORT_THREADS;
static_assert(SORT_VPT % 4 == 0, "vector loads of keys and payloads");

__device__ __forceinline__ void load_run(const uint32_t* __restrict__ a, int64_t e0, uint32_t (&v)[SORT_VPT])
{
    const uint4* a4 = reinterpret_cast<const uint4*>(a + e0);
#pragma unroll
    for (int q = 0; q < SORT_VPT / 4; ++q) {
        const uint4 x = __ldg(a4 + q);
        v[4 * q + 0] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
    }
}

// fixed-point sums of (w, w a) over the sources of each sorted tile; thread j
// takes the tile's elements SORT_VPT j .. SORT_VPT (j + 1) - 1 (the buffers
// hold whole tiles, so the vector loads stay inside them; elements >= L are
// skipped)
__global__ void __launch_bounds__(SORT_THREADS) sort_tilesum_kernel(const uint32_t* __restrict__ key,
                                                                    const uint32_t* __restrict__ pay, int64_t N,
                                                                    int64_t L, int64_t LS, int T,
                                                                    const float* __restrict__ w,
                                                                    const SortScale* __restrict__ scp,
                                                                    long long* __restrict__ tsum)
{
    __shared__ long long rw[SORT_THREADS / 32], ra[SORT_THREADS / 32];
    const int t = blockIdx.x, pl = blockIdx.y;
    const uint32_t* k = key + (size_t)pl * LS;
    const uint32_t* p = pay + (size_t)pl * LS;
    const SliceScale sc = slice_scale(scp, w == nullptr, N, k, L);
    const int64_t e0 = (int64_t)t * SORT_TILE + (int64_t)threadIdx.x * SORT_VPT;
    uint32_t kk[SORT_VPT], pp[SORT_VPT];
    load_run(k, e0, kk);
    load_run(p, e0, pp);
    long long sw = 0, sa = 0;
#pragma unroll
    for (int j = 0; j < SORT_VPT; ++j) {
        if (e0 + j < L && pp[j] < N) {
            long long qw, qs;
            src_fixed(w ? __ldg(&w[pp[j]]) : 1.0f, key_float(kk[j]), sc, qw, qs);
            sw += qw;
            sa += qs;
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
        long long tw = 0, ta = 0;
        for (int q = 0; q < SORT_THREADS / 32; ++q) {
            tw += rw[q];
            ta += ra[q];
        }
        tsum[((size_t)pl * T + t) * 2 + 0] = tw;
        tsum[((size_t)pl * T + t) * 2 + 1] = ta;
    }
}

// per slice (one warp each, 32 tiles at a time): exclusive prefix of the tile
// sums in place, totals in tot[pl] (integer sums: exact in any order)
__global__ void sort_tilescan_kernel(long long* __restrict__ tsum, int T, int cs, long long* __restrict__ tot)
{
    const int pl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (pl >= cs) return;  // whole warps
    long long* ts = tsum + (size_t)pl * T * 2;
    long long rw = 0, ra = 0;
    for (int t0 = 0; t0 < T; t0 += 32) {
        const int t = t0 + lane;
        const long long cw = t < T ? ts[2 * t] : 0, ca = t < T ? ts[2 * t + 1] : 0;
        long long iw = cw, ia = ca;
        for (int o = 1; o < 32; o <<= 1) {
            const long long nw = __shfl_up_sync(0xffffffffu, iw, o);
            const long long na = __shfl_up_sync(0xffffffffu, ia, o);
            if (lane >= o) {
                iw += nw;
                ia += na;
            }
        }
        if (t < T) {
            ts[2 * t] = rw + iw - cw;
            ts[2 * t + 1] = ra + ia - ca;
        }
        rw += __shfl_sync(0xffffffffu, iw, 31);
        ra += __shfl_sync(0xffffffffu, ia, 31);
    }
    if (lane == 0) {
        tot[2 * pl] = rw;
        tot[2 * pl + 1] = ra;
    }
}

// per sorted tile (elements per thread as in the tile sums): the fixed-point
// prefix of (w, w a) over the sources before each element; for every target m
// the slice's value b (2 W_< - W) - (2 S_< - S) goes to t[pl][m] (the factor
// of the kernel and the grid is applied once per target at the end)
// GRAD: t[pl][m] = 2 W_< - W = sum_n w_n sign(b - a_n) instead (sources whose
// projection equals b count as below).
template <bool GRAD>
__global__ void __launch_bounds__(SORT_THREADS, 4) sort_eval_kernel(const uint32_t* __restrict__ key,
                                                                 const uint32_t* __restrict__ pay, int64_t N,
                                                                 int64_t M, int64_t LS, int T,
                                                                 const float* __restrict__ w,
                                                                 const SortScale* __restrict__ scp,
                                                                 const long long* __restrict__ tsum,
                                                                 const long long* __restrict__ tot,
                                                                 float* __restrict__ tout)
{
    __shared__ long long sw[SORT_THREADS / 32], sa[SORT_THREADS / 32];
    const int t = blockIdx.x, pl = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t* k = key + (size_t)pl * LS;
    const uint32_t* p = pay + (size_t)pl * LS;
    const int64_t L = N + M;
    const SliceScale sc = slice_scale(scp, w == nullptr, N, k, L);
    const int64_t e0 = (int64_t)t * SORT_TILE + (int64_t)threadIdx.x * SORT_VPT;
    uint32_t kk[SORT_VPT], pp[SORT_VPT];
    load_run(k, e0, kk);
    load_run(p, e0, pp);
    long long qw[SORT_VPT], qs[SORT_VPT];
    long long tw = 0, ta = 0;
#pragma unroll
    for (int j = 0; j < SORT_VPT; ++j) {
        qw[j] = 0;
        qs[j] = 0;
        if (e0 + j < L && pp[j] < N)
            src_fixed(w ? __ldg(&w[pp[j]]) : 1.0f, key_float(kk[j]), sc, qw[j], qs[j]);
        tw += qw[j];
        ta += qs[j];
    }
    long long iw = tw, ia = ta;  // inclusive warp scan of the threads' sums
    for (int o = 1; o < 32; o <<= 1) {
        const long long nw = __shfl_up_sync(0xffffffffu, iw, o);
        const long long na = __shfl_up_sync(0xffffffffu, ia, o);
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
    long long ow = tsum[((size_t)pl * T + t) * 2 + 0] + iw - tw;
    long long oa = tsum[((size_t)pl * T + t) * 2 + 1] + ia - ta;
    for (int q = 0; q < warp; ++q) {
        ow += sw[q];
        oa += sa[q];
    }
    const long long W = tot[2 * pl], S = tot[2 * pl + 1];
#pragma unroll
    for (int j = 0; j < SORT_VPT; ++j) {
        // sources strictly before (a target contributes nothing of its own)
        if (e0 + j < L && pp[j] >= N) {
            const long long XW = 2 * ow - W;
            float v;
            if (GRAD) {
                float hi, lo;
                split_fixed(XW, hi, lo);
                v = (hi + lo) * sc.g1 * sc.g2;
            } else {
                v = sorted_value(key_float(kk[j]), XW, 2 * oa - S, sc);
            }
            tout[(size_t)pl * M + (pp[j] - N)] = v;
        }
        ow += qw[j];
        oa += qs[j];
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

// s[m] = amp (hi + lo) / P: the factor of the kernel and the grid, once per target
__global__ void sort_final_kernel(const float* __restrict__ hi, const float* __restrict__ lo, int64_t M,
                                  double amp_p, float* __restrict__ s)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) s[m] = (float)(((double)hi[m] + (double)lo[m]) * amp_p);
}

}  // namespace

// Chunk of slices and the workspace for up to L = N + M points.
int qs_sort_chunk(int P) { return P < 128 ? P : 128; }

size_t qs_sort_workspace_bytes(int P, int64_t max_n, int64_t max_m)
{
    const int CS = qs_sort_chunk(P);
    const int64_t L = max_n + max_m;
    const int64_t LS = (L + SORT_TILE - 1) / SORT_TILE * SORT_TILE;
    const int64_t T = LS / SORT_TILE;
    const int64_t PR = (max_n + 127) / 128 * 128 + (max_m + 127) / 128 * 128;
    return (size_t)4 * CS * LS * sizeof(uint32_t)         // key / payload, two buffers each
           + (size_t)CS * PR * sizeof(float)              // projections of a chunk
           + (size_t)CS * 256 * T * sizeof(uint32_t)      // digit offsets
           + (size_t)CS * T * 2 * sizeof(long long)       // tile sums (fixed point)
           + (size_t)CS * 2 * sizeof(long long)           // slice totals
           + 64                                           // max |w|
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
    long long* tsum = reinterpret_cast<long long*>(hist + (size_t)CS * 256 * Tmax);  // 8-byte aligned: even count
    long long* tot = tsum + (size_t)CS * Tmax * 2;
    SortScale* scale_rec = reinterpret_cast<SortScale*>(tot + (size_t)CS * 2);
    float* tb = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(scale_rec) + 64);
    float* hi = tb + (size_t)CS * max_m;
    float* lo = hi + max_m;
    // the chunk's projections after the accumulators (at most 2 max_m d floats), on a 256-byte
    // boundary inside the workspace's 1 KB of slack (the GEMM stores 16-byte vectors)
    const int64_t ldp = (max_n + 127) / 128 * 128 + (max_m + 127) / 128 * 128;
    const int64_t Nr = (N + 127) / 128 * 128;
    float* proj = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(hi + (size_t)2 * max_m * QS_FUSED_MAX_D) + 255) & ~(uintptr_t)255);
    const size_t acc = (size_t)M * (grad ? d : 1);  // accumulators of this call, hi then lo
    lo = hi + acc;
    cudaError_t e = cudaMemsetAsync(hi, 0, sizeof(float) * 2 * acc, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scale_rec, 0, sizeof(SortScale), st);
    if (e == cudaSuccess && w && N > 0) {
        const int64_t nb = (N + 255) / 256;
        sort_wmax_kernel<<<(unsigned)(nb < 2 * 152 ? nb : 2 * 152), 256, 0, st>>>(w, N, scale_rec, flag);
        e = cudaGetLastError();
    }
    for (int p0 = 0; p0 < P && e == cudaSuccess; p0 += CS) {
        const int cs = P - p0 < CS ? P - p0 : CS;
        if (N > 0) e = qs_launch_project_fp32(x, N, d, xi_s + (size_t)p0 * d, cs, proj, ldp, st);
        if (e == cudaSuccess) e = qs_launch_project_fp32(y, M, d, xi_s + (size_t)p0 * d, cs, proj + Nr, ldp, st);
        if (e != cudaSuccess) break;
        // pass 0 reads the projections and writes A; then A -> B -> A -> B
        uint32_t *ki = kB, *pi = pB, *ko = kA, *po = pA;
        const dim3 tg((unsigned)T, (unsigned)cs);
        for (int shift = 0; shift < 32; shift += 8) {
            const KeySrc ks{ki, pi, proj, N, Nr, ldp, flag};
            if (shift == 0) sort_hist_kernel<true><<<tg, SORT_THREADS, 0, st>>>(ks, L, LS, T, shift, hist);
            else sort_hist_kernel<false><<<tg, SORT_THREADS, 0, st>>>(ks, L, LS, T, shift, hist);
            sort_scan_kernel<<<cs, 1024, 0, st>>>(hist, T);
            if (shift == 0) sort_scatter_kernel<true><<<tg, SORT_THREADS, 0, st>>>(ks, L, LS, T, shift, hist, ko, po);
            else sort_scatter_kernel<false><<<tg, SORT_THREADS, 0, st>>>(ks, L, LS, T, shift, hist, ko, po);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            uint32_t* tk = ki;
            ki = ko;
            ko = tk;
            tk = pi;
            pi = po;
            po = tk;
        }
        if (e != cudaSuccess) break;
        // four passes: the sorted data are in the B buffers (ki, pi)
        sort_tilesum_kernel<<<dim3((unsigned)T, (unsigned)cs), SORT_THREADS, 0, st>>>(ki, pi, N, L, LS, T, w,
                                                                                     scale_rec, tsum);
        sort_tilescan_kernel<<<(unsigned)((cs + 7) / 8), 256, 0, st>>>(tsum, T, cs, tot);
        const dim3 eg((unsigned)T, (unsigned)cs);
        if (grad) {
            sort_eval_kernel<true><<<eg, SORT_THREADS, 0, st>>>(ki, pi, N, M, LS, T, w, scale_rec, tsum, tot, tb);
            sort_gaccum_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(tb, cs, M, xi, d, p0, hi, lo);
        } else {
            sort_eval_kernel<false><<<eg, SORT_THREADS, 0, st>>>(ki, pi, N, M, LS, T, w, scale_rec, tsum, tot, tb);
            sort_accum_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(tb, cs, M, hi, lo);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (grad)
            sort_gfinal_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(hi, lo, M, d, v, scale, gy);
        else
            sort_final_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(hi, lo, M, amp / P, s);
        e = cudaGetLastError();
    }
    return e;
}
