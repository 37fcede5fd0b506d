// Batched sums: many independent problems (each with its own plan: d, P,
// N_ft, kernel, directions) of uneven N and M in one persistent launch.
//
// Work items, dequeued in order from one 64-bit counter:
//   projection items     (problem k, x or y, 128-slice x 128-point tile): the
//                        FP32 SIMT projection tile U = G tau Xi X^T into the
//                        batch's per-problem projection buffers
//   spread items         (problem k, slice p): spread + FFT filter of slice p,
//                        writing the problem's filtered grid row H_k[p]
//   interpolation items  (problem k, target block b): interpolation of a block
//                        of targets over all P_k slices, writing s directly
// Problems are queued largest first within each phase.  A spread item waits
// for its problem's x-projection tiles; an interpolation item waits for all
// P_k spread items and the y-projection tiles of its problem (per-problem
// counters, incremented after a fence).  Every awaited item was dequeued
// earlier, so it is held by a running CTA and will finish: no wait can
// deadlock, whatever the grid size.  Waits are bounded by a clock budget; on
// expiry the item sets the problem's timeout flag and is skipped.  Data
// written in this launch is read back through L2 only (ld.global.cg /
// cp.async.cg).
//
// Problems with d <= 4 skip the projection items and form their dot products
// inside the spread and interpolation items (the fused form is cheaper when
// a point has so few coordinates).  Each target's slice sum runs in slice
// order with TwoSum in one thread, so the result does not depend on the
// tiling chosen by the tuner.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.cuh"

using namespace qsdev;

namespace {

constexpr int BT = 256;                  // threads per CTA
constexpr int FUSED_MAX_D = 4;           // problems with d <= 4 use fused projections
constexpr int YTILE_BYTES = BT * 4 * FUSED_MAX_D * 4;  // coordinate tile of a fused block
constexpr int GEMM_SMEM = 4 * GT_BK * GT_BM * 4;       // 16 KB

struct BatchDesc {
    const float* x;
    const float* w;
    const float* y;
    float* s;
    int64_t N, M;
    int d, P, G, tpt;
    int fused, vecx, vecy;
    float half_G;
    const float* xi_s;
    const float* D;
    const float2* tw;
    float* H;
    float* Ux;            // P x ldUx projections of x (unfused problems)
    float* Uy;            // P x ldUy projections of y
    int64_t ldUx, ldUy;
    int ptiles;           // ceil(P / 128)
    int64_t nxt, nyt;     // projection tiles of x and y
    unsigned int* flag;
    int64_t proj_begin, spread_begin, interp_begin, interp_blocks;
};

// last problem k whose phase-`ph` range begins at or before `item`
// (ph: 0 projection, 1 spread, 2 interpolation)
__device__ int find_item(const BatchDesc* __restrict__ descs, int nprob, int64_t item, int ph)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t b = ph == 0 ? descs[mid].proj_begin : (ph == 1 ? descs[mid].spread_begin : descs[mid].interp_begin);
        if (b <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Spin (thread 0) until *ctr >= target or the clock budget is spent.
__device__ bool wait_count(unsigned int* ctr, unsigned int target, long long budget, unsigned int* flag)
{
    const long long t0 = clock64();
    while (atomicAdd(ctr, 0u) < target) {
        if (clock64() - t0 > budget) {
            atomicOr(flag, QS_FLAG_TIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
    __threadfence();
    return true;
}

template <int W>
__device__ void batch_spread(const BatchDesc& D, int p, const qs_window& win, unsigned char* smem)
{
    __shared__ float xi_sm[QS_BATCH_MAX_D];
    __shared__ float red[BT / 32];
    __shared__ float s_scale[2];
    int* gridi = reinterpret_cast<int*>(smem);
    float* grid = reinterpret_cast<float*>(smem);
    const int G = D.G, mask = G - 1, d = D.d;
    for (int i = threadIdx.x; i < G; i += BT) gridi[i] = 0;
    for (int j = threadIdx.x; j < d; j += BT) xi_sm[j] = __ldg(&D.xi_s[(size_t)p * d + j]);
    // fixed-point scale 2^30 / sum|w| (as in the single-problem spread)
    float acc = 0.0f;
    if (D.w)
        for (int64_t n = threadIdx.x; n < D.N; n += BT) acc += fabsf(__ldg(&D.w[n]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float B = 0.0f;
        for (int i = 0; i < BT / 32; ++i) B += red[i];
        if (!D.w) B = (float)D.N;
        float sc = 0.0f, inv = 0.0f;
        if (!isfinite(B)) {
            atomicOr(D.flag, QS_FLAG_NONFINITE);
        } else if (B > 0.0f) {
            sc = 1073741824.0f / B;
            inv = B / 1073741824.0f;
            if (!isfinite(sc)) sc = inv = 0.0f;
        }
        s_scale[0] = sc;
        s_scale[1] = inv;
    }
    __syncthreads();
    const float scale = s_scale[0];
    const float* urow = D.Ux + (size_t)p * D.ldUx;
    for (int64_t n = threadIdx.x; n < D.N; n += BT) {
        float u;
        if (D.fused) {
            const float* xn = D.x + (size_t)n * d;
            u = 0.0f;
            for (int j = 0; j < d; ++j) u = fmaf(xi_sm[j], __ldg(&xn[j]), u);
        } else {
            u = __ldcg(&urow[n]);  // written by projection items of this launch
        }
        u = qs_check_u(u, D.half_G, D.flag);
        float wn = D.w ? __ldg(&D.w[n]) : 1.0f;
        if (!isfinite(wn)) {
            atomicOr(D.flag, QS_FLAG_NONFINITE);
            wn = 0.0f;
        }
        const float ws = wn * scale;
        int l0;
        float tap[W];
        qs_taps<W>(u, win, l0, tap);
#pragma unroll
        for (int j = 0; j < W; ++j) atomicAdd(&gridi[(l0 + j) & mask], __float2int_rn(ws * tap[j]));
    }
    __syncthreads();
    const float inv_scale = s_scale[1];
    for (int i = threadIdx.x; i < G; i += BT) grid[i] = (float)gridi[i] * inv_scale;
    __syncthreads();
    const int Gh = G >> 1;
    const int log2n = 31 - __clz(Gh);
    float2* z = reinterpret_cast<float2*>(grid);
    fft_inplace<false>(z, Gh, log2n, D.tw, G);
    real_filter<false>(z, Gh, D.D, D.tw);
    __syncthreads();
    fft_inplace<true>(z, Gh, log2n, D.tw, G);
    float4* dst = reinterpret_cast<float4*>(D.H + (size_t)p * G);
    const float4* src = reinterpret_cast<const float4*>(grid);
    for (int i = threadIdx.x; i < (G >> 2); i += BT) dst[i] = src[i];
}

template <int W>
__device__ void batch_interp(const BatchDesc& D, int64_t b, const qs_window& win, unsigned char* smem)
{
    const int d = D.d, G = D.G, mask = G - 1, tpt = D.tpt;
    const int TB = BT * tpt;
    const int64_t m0 = b * TB;
    float* ytile = reinterpret_cast<float*>(smem);                  // [d][TB]
    float* rows = reinterpret_cast<float*>(smem + YTILE_BYTES);     // 2 x (G + ROW_PAD)
    const int stride = G + ROW_PAD;
    if (D.fused) {
        const int64_t nload = (int64_t)TB * d;
        for (int64_t i = threadIdx.x; i < nload; i += BT) {
            const int t = (int)(i / d), j = (int)(i - (int64_t)t * d);
            const int64_t m = m0 + t;
            ytile[j * TB + t] = m < D.M ? __ldg(&D.y[(size_t)m * d + j]) : 0.0f;
        }
    }
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    const int P = D.P;
    stage_row(rows, D.H, G);
    for (int p = 0; p < P; ++p) {
        const float* row = rows + (p & 1) * stride;
        if (p + 1 < P) {
            stage_row(rows + ((p + 1) & 1) * stride, D.H + (size_t)(p + 1) * G, G);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* xs = D.xi_s + (size_t)p * d;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i >= tpt) break;
            const int t = threadIdx.x + i * BT;
            if (m0 + t >= D.M) continue;
            float u;
            if (D.fused) {
                u = 0.0f;
                for (int j = 0; j < d; ++j) u = fmaf(__ldg(&xs[j]), ytile[j * TB + t], u);
            } else {
                u = __ldcg(&D.Uy[(size_t)p * D.ldUy + m0 + t]);
            }
            u = qs_check_u(u, D.half_G, D.flag);
            int l0;
            float tap[W];
            qs_taps<W>(u, win, l0, tap);
            const float* h = row + (l0 & mask);
            float v = 0.0f;
#pragma unroll
            for (int j = 0; j < W; ++j) v = fmaf(h[j], tap[j], v);
            qs_two_sum(hi[i], lo[i], v);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i >= tpt) break;
        const int64_t m = m0 + threadIdx.x + i * BT;
        if (m < D.M) D.s[m] = (hi[i] + lo[i]) / (float)P;
    }
}

template <int W>
__global__ void __launch_bounds__(BT, 2)
    batched_kernel(const BatchDesc* __restrict__ descs, int nprob, int64_t n_proj, int64_t n_spread, int64_t n_items,
                   unsigned long long* __restrict__ counter, unsigned int* __restrict__ done, qs_window win,
                   long long wait_cycles)
{
    // done[0..n): spread rows published, [n..2n): x tiles, [2n..3n): y tiles
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    __shared__ long long s_item;
    __shared__ int s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= n_items) return;
        if (item < n_proj) {
            const int k = find_item(descs, nprob, item, 0);
            const BatchDesc D = descs[k];
            int64_t j = item - D.proj_begin;
            const bool isx = j < D.nxt;
            if (!isx) j -= D.nxt;
            const int p0 = (int)(j % D.ptiles) * GT_BM;
            const int64_t n0 = (j / D.ptiles) * GT_BN;
            float* sm = reinterpret_cast<float*>(smem);
            if (isx) {
                if (D.vecx) gemm_tile_fp32<true>(D.x, D.N, D.d, D.xi_s, D.P, D.Ux, D.ldUx, p0, n0, sm);
                else gemm_tile_fp32<false>(D.x, D.N, D.d, D.xi_s, D.P, D.Ux, D.ldUx, p0, n0, sm);
            } else {
                if (D.vecy) gemm_tile_fp32<true>(D.y, D.M, D.d, D.xi_s, D.P, D.Uy, D.ldUy, p0, n0, sm);
                else gemm_tile_fp32<false>(D.y, D.M, D.d, D.xi_s, D.P, D.Uy, D.ldUy, p0, n0, sm);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&done[(isx ? 1 : 2) * nprob + k], 1u);
        } else if (item < n_spread) {
            const int k = find_item(descs, nprob, item, 1);
            const BatchDesc D = descs[k];
            if (threadIdx.x == 0) s_ok = wait_count(&done[nprob + k], (unsigned)D.nxt, wait_cycles, D.flag);
            __syncthreads();
            if (s_ok) {
                batch_spread<W>(D, (int)(item - D.spread_begin), win, smem);
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) atomicAdd(&done[k], 1u);
            }
        } else {
            const int k = find_item(descs, nprob, item, 2);
            const BatchDesc D = descs[k];
            if (threadIdx.x == 0) {
                s_ok = wait_count(&done[k], (unsigned)D.P, wait_cycles, D.flag) &&
                       wait_count(&done[2 * nprob + k], (unsigned)D.nyt, wait_cycles, D.flag);
            }
            __syncthreads();
            if (s_ok) batch_interp<W>(D, item - D.interp_begin, win, smem);
        }
        __syncthreads();
    }
}

qs_status bfail(qs_status st, const char* fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    qs_set_error_message(msg);
    return st;
}

}  // namespace

struct qs_batch_s {
    int device;
    int sm_count;
    int nprob;
    int W;
    int tpt_cap;            // largest targets-per-thread of interpolation items (1, 2 or 4)
    qs_window win;
    std::vector<qs_plan> plans;
    std::vector<float*> Ux, Uy;     // per-problem projection buffers (d > 4)
    std::vector<int64_t> ldUx, ldUy;
    BatchDesc* h_desc;      // pinned host staging of the descriptors
    cudaEvent_t uploaded;   // recorded after each upload of h_desc
    BatchDesc* d_desc;
    unsigned long long* d_counter;
    unsigned int* d_done;   // 3 counters per problem
    // concurrent mode: every problem's own pipeline (qs_sum) on one of the
    // batch's streams, forked from and joined to the caller's stream
    int mode;               // QS_BATCH_PERSISTENT or QS_BATCH_CONCURRENT
    cudaStream_t st[QS_BATCH_STREAMS];
    cudaEvent_t fork_ev;
    cudaEvent_t join_ev[QS_BATCH_STREAMS];
};

extern "C" qs_status qs_batch_destroy(qs_batch b);

extern "C" qs_status qs_batch_create(qs_batch* out, const qs_plan* plans, int nprob)
{
    if (!out || !plans || nprob < 1) return bfail(QS_ERR_ARG, "qs_batch_create: bad arguments");
    *out = nullptr;
    const int dev = plans[0] ? plans[0]->device : -1;
    for (int k = 0; k < nprob; ++k) {
        const qs_plan p = plans[k];
        if (!p) return bfail(QS_ERR_ARG, "qs_batch_create: plan %d is NULL", k);
        if (p->device != dev) return bfail(QS_ERR_ARG, "qs_batch_create: plans on different devices");
        if (p->W != plans[0]->W || p->window_kind != plans[0]->window_kind)
            return bfail(QS_ERR_UNSUPPORTED, "qs_batch_create: plans must share the window (width and kind)");
        if (p->desc.d > QS_BATCH_MAX_D)
            return bfail(QS_ERR_UNSUPPORTED, "qs_batch_create: d = %d exceeds %d", p->desc.d, QS_BATCH_MAX_D);
        for (int j = 0; j < k; ++j)
            if (plans[j] == p) return bfail(QS_ERR_ARG, "qs_batch_create: plan %d repeated (plans hold the grids)", k);
    }
    qs_batch b = new (std::nothrow) qs_batch_s;
    if (!b) return bfail(QS_ERR_OOM, "qs_batch_create: host allocation");
    b->device = dev;
    b->sm_count = plans[0]->sm_count;
    b->nprob = nprob;
    b->W = plans[0]->W;
    b->tpt_cap = 4;
    b->win = plans[0]->win;
    b->plans.assign(plans, plans + nprob);
    b->Ux.assign(nprob, nullptr);
    b->Uy.assign(nprob, nullptr);
    b->ldUx.assign(nprob, 0);
    b->ldUy.assign(nprob, 0);
    b->h_desc = nullptr;
    b->uploaded = nullptr;
    b->d_desc = nullptr;
    b->d_counter = nullptr;
    b->d_done = nullptr;
    b->mode = QS_BATCH_PERSISTENT;
    b->fork_ev = nullptr;
    for (int i = 0; i < QS_BATCH_STREAMS; ++i) {
        b->st[i] = nullptr;
        b->join_ev[i] = nullptr;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    cudaError_t e = cudaMallocHost((void**)&b->h_desc, sizeof(BatchDesc) * nprob);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_desc, sizeof(BatchDesc) * nprob);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_done, sizeof(unsigned int) * 3 * nprob);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < QS_BATCH_STREAMS && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming);
    }
    for (int k = 0; k < nprob && e == cudaSuccess; ++k) {
        const qs_plan p = plans[k];
        if (p->desc.d <= FUSED_MAX_D) continue;
        b->ldUx[k] = ((p->desc.max_n > 0 ? p->desc.max_n : 1) + 127) / 128 * 128;
        b->ldUy[k] = ((p->desc.max_m > 0 ? p->desc.max_m : 1) + 127) / 128 * 128;
        e = cudaMalloc((void**)&b->Ux[k], sizeof(float) * (size_t)p->desc.P * b->ldUx[k]);
        if (e == cudaSuccess) e = cudaMalloc((void**)&b->Uy[k], sizeof(float) * (size_t)p->desc.P * b->ldUy[k]);
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        qs_batch_destroy(b);
        return bfail(QS_ERR_OOM, "qs_batch_create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return QS_OK;
}

extern "C" qs_status qs_batch_destroy(qs_batch b)
{
    if (!b) return QS_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->h_desc) cudaFreeHost(b->h_desc);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_done) cudaFree(b->d_done);
    if (b->uploaded) cudaEventDestroy(b->uploaded);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (int i = 0; i < QS_BATCH_STREAMS; ++i) {
        if (b->st[i]) cudaStreamDestroy(b->st[i]);
        if (b->join_ev[i]) cudaEventDestroy(b->join_ev[i]);
    }
    for (float* u : b->Ux)
        if (u) cudaFree(u);
    for (float* u : b->Uy)
        if (u) cudaFree(u);
    cudaSetDevice(prev);
    delete b;
    return QS_OK;
}

extern "C" qs_status qs_batch_set_mode(qs_batch b, int mode)
{
    if (!b || (mode != QS_BATCH_PERSISTENT && mode != QS_BATCH_CONCURRENT))
        return bfail(QS_ERR_ARG, "qs_batch_set_mode: bad value");
    b->mode = mode;
    return QS_OK;
}

extern "C" qs_status qs_batch_set_tiling(qs_batch b, int tpt_cap)
{
    if (!b || (tpt_cap != 1 && tpt_cap != 2 && tpt_cap != 4)) return bfail(QS_ERR_ARG, "qs_batch_set_tiling: bad value");
    b->tpt_cap = tpt_cap;
    return QS_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Concurrent mode: problems, largest first, each go to the batch stream with
// the least work queued so far (longest-processing-time list scheduling by
// (N + M) P) and run their own plan's qs_sum there; the streams wait for the
// work already on `stream` and `stream` waits for all of them, so the call is
// ordered like any other on `stream` and can be captured into a CUDA graph
// (the fork and join become graph dependencies).
static qs_status batched_concurrent(qs_batch b, const qs_problem* probs, const std::vector<int>& order,
                                    cudaStream_t stream)
{
    double load[QS_BATCH_STREAMS] = {0.0};
    bool used[QS_BATCH_STREAMS] = {false};
    cudaError_t e = cudaEventRecord(b->fork_ev, stream);
    for (size_t i = 0; i < order.size() && e == cudaSuccess; ++i) {
        const int k = order[i];
        const qs_problem& q = probs[k];
        int si = 0;
        for (int j = 1; j < QS_BATCH_STREAMS; ++j)
            if (load[j] < load[si]) si = j;
        if (!used[si]) {
            e = cudaStreamWaitEvent(b->st[si], b->fork_ev, 0);
            if (e != cudaSuccess) break;
            used[si] = true;
        }
        load[si] += (double)(q.N + q.M) * b->plans[k]->desc.P + 1e6;  // + a launch-overhead term
        const qs_status s = qs_sum(b->plans[k], q.x, q.N, q.w, q.y, q.M, q.s, b->st[si]);
        if (s != QS_OK) return s;
    }
    for (int j = 0; j < QS_BATCH_STREAMS && e == cudaSuccess; ++j) {
        if (!used[j]) continue;
        e = cudaEventRecord(b->join_ev[j], b->st[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->join_ev[j], 0);
    }
    if (e != cudaSuccess) return bfail(QS_ERR_CUDA, "qs_sum_batched: %s", cudaGetErrorString(e));
    return QS_OK;
}

extern "C" qs_status qs_sum_batched(qs_batch b, const qs_problem* probs, void* stream)
{
    if (!b || !probs) return bfail(QS_ERR_ARG, "qs_sum_batched: NULL argument");
    const int n = b->nprob;
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) {
        const qs_problem& q = probs[k];
        const qs_plan p = b->plans[k];
        if (q.N < 0 || q.M < 0 || q.N > p->desc.max_n || q.M > p->desc.max_m)
            return bfail(QS_ERR_ARG, "qs_sum_batched: problem %d sizes outside its plan's limits", k);
        if ((q.N > 0 && !q.x) || (q.M > 0 && (!q.y || !q.s)))
            return bfail(QS_ERR_ARG, "qs_sum_batched: problem %d has a NULL data pointer", k);
        order[k] = k;
    }
    // queue order: largest problems first
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const double wa = (double)(probs[a].N + probs[a].M) * b->plans[a]->desc.P;
        const double wc = (double)(probs[c].N + probs[c].M) * b->plans[c]->desc.P;
        return wa > wc;
    });
    if (b->mode == QS_BATCH_CONCURRENT) return batched_concurrent(b, probs, order, (cudaStream_t)stream);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const double wa = (double)(probs[a].N + probs[a].M) * b->plans[a]->desc.P;
        const double wc = (double)(probs[c].N + probs[c].M) * b->plans[c]->desc.P;
        return wa > wc;
    });
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return bfail(QS_ERR_CUDA, "qs_sum_batched: stream query");
    if (cap == cudaStreamCaptureStatusNone && cudaEventSynchronize(b->uploaded) != cudaSuccess)
        return bfail(QS_ERR_CUDA, "qs_sum_batched: previous upload");
    int64_t proj_items = 0, spread_items = 0, interp_items = 0;
    int maxG = 32;
    for (int i = 0; i < n; ++i) {
        const int k = order[i];
        const qs_problem& q = probs[k];
        const qs_plan p = b->plans[k];
        BatchDesc& D = b->h_desc[i];
        D.x = q.x;
        D.w = q.w;
        D.y = q.y;
        D.s = q.s;
        D.N = q.N;
        D.M = q.M;
        D.d = p->desc.d;
        D.P = p->desc.P;
        D.G = p->G;
        D.fused = D.d <= FUSED_MAX_D ? 1 : 0;
        D.vecx = (D.d % 4 == 0) && aligned16(q.x) && aligned16(p->d_dirs_s);
        D.vecy = (D.d % 4 == 0) && aligned16(q.y) && aligned16(p->d_dirs_s);
        D.tpt = b->tpt_cap;
        D.half_G = 0.5f * (float)p->G;
        D.xi_s = p->d_dirs_s;
        D.D = p->d_D;
        D.tw = p->d_tw;
        D.H = p->d_H;
        D.Ux = b->Ux[k];
        D.Uy = b->Uy[k];
        D.ldUx = b->ldUx[k];
        D.ldUy = b->ldUy[k];
        D.ptiles = (D.P + GT_BM - 1) / GT_BM;
        D.nxt = D.fused ? 0 : (int64_t)D.ptiles * ((q.N + GT_BN - 1) / GT_BN);
        D.nyt = D.fused ? 0 : (int64_t)D.ptiles * ((q.M + GT_BN - 1) / GT_BN);
        if (q.M == 0) D.nxt = D.nyt = 0;  // nothing to compute for this problem
        D.flag = p->d_flag;
        D.proj_begin = proj_items;
        proj_items += D.nxt + D.nyt;
        D.spread_begin = spread_items;  // made absolute below
        spread_items += q.M > 0 ? D.P : 0;
        D.interp_begin = interp_items;
        D.interp_blocks = q.M > 0 ? (q.M + (int64_t)BT * D.tpt - 1) / ((int64_t)BT * D.tpt) : 0;
        interp_items += D.interp_blocks;
        if (p->G > maxG) maxG = p->G;
    }
    for (int i = 0; i < n; ++i) {
        b->h_desc[i].spread_begin += proj_items;
        b->h_desc[i].interp_begin += proj_items + spread_items;
    }
    const int64_t n_proj = proj_items;
    const int64_t n_spread_end = proj_items + spread_items;
    const int64_t n_items = n_spread_end + interp_items;
    if (n_items == 0) return QS_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(BatchDesc) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && cap == cudaStreamCaptureStatusNone) e = cudaEventRecord(b->uploaded, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * 3 * n, st);
    // shared memory: the union of a projection tile, a spread grid, and an
    // interpolation block (fused coordinate tile + two staged rows)
    size_t smem = (size_t)YTILE_BYTES + (size_t)2 * (maxG + ROW_PAD) * sizeof(float);
    if ((size_t)maxG * 4 > smem) smem = (size_t)maxG * 4;
    if ((size_t)GEMM_SMEM > smem) smem = GEMM_SMEM;
    const long long wait_cycles = 4000000000LL;  // ~2 s at 2 GHz
    const unsigned grid = (unsigned)(b->sm_count * 2);
#define QS_BATCH_LAUNCH(WW)                                                                                   \
    do {                                                                                                      \
        if (e == cudaSuccess)                                                                                 \
            e = cudaFuncSetAttribute(batched_kernel<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess) {                                                                               \
            batched_kernel<WW><<<grid, BT, smem, st>>>(b->d_desc, n, n_proj, n_spread_end, n_items, b->d_counter, \
                                                       b->d_done, b->win, wait_cycles);                      \
            e = cudaGetLastError();                                                                           \
        }                                                                                                     \
    } while (0)
    switch (b->W) {
        case 6: QS_BATCH_LAUNCH(6); break;
        case 8: QS_BATCH_LAUNCH(8); break;
        case 10: QS_BATCH_LAUNCH(10); break;
        case 12: QS_BATCH_LAUNCH(12); break;
        default: e = cudaErrorInvalidValue;
    }
#undef QS_BATCH_LAUNCH
    if (prev != b->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(QS_ERR_CUDA, "qs_sum_batched: %s", cudaGetErrorString(e));
    return QS_OK;
}

extern "C" qs_status qs_batch_check(qs_batch b, void* stream)
{
    if (!b) return bfail(QS_ERR_ARG, "qs_batch_check: NULL batch");
    qs_status worst = QS_OK;
    for (int k = 0; k < b->nprob; ++k) {
        const qs_status s = qs_check(b->plans[k], stream);
        if (s != QS_OK && (worst == QS_OK || s == QS_ERR_CUDA || s == QS_ERR_TIMEOUT)) worst = s;
    }
    return worst;
}

// Time the batched sum of these problems with the persistent kernel at each
// interpolation tiling (1, 2 and 4 targets per thread) and in the concurrent
// mode (best of two after a warm-up, CUDA events on `stream`) and keep the
// fastest.  The tilings give the same bits; the concurrent mode gives each
// plan's own qs_sum result.
extern "C" qs_status qs_batch_autotune(qs_batch b, const qs_problem* probs, int* chosen, void* stream)
{
    if (!b || !probs) return bfail(QS_ERR_ARG, "qs_batch_autotune: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return bfail(QS_ERR_CUDA, "qs_batch_autotune: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(QS_ERR_CUDA, "qs_batch_autotune: event");
    }
    const int keep = b->tpt_cap, keep_mode = b->mode;
    int best = keep_mode == QS_BATCH_CONCURRENT ? 0 : keep;
    float best_ms = 3.4e38f;
    qs_status s = QS_OK;
    // tpt 1, 2, 4: the persistent kernel with that tiling; 0 (tried last): concurrent pipelines
    for (int tpt = 1; tpt <= 8 && s == QS_OK; tpt *= 2) {
        b->mode = tpt == 8 ? QS_BATCH_CONCURRENT : QS_BATCH_PERSISTENT;
        if (tpt < 8) b->tpt_cap = tpt;
        s = qs_sum_batched(b, probs, stream);  // warm-up
        float tb = 3.4e38f;
        for (int r = 0; r < 2 && s == QS_OK; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) s = QS_ERR_CUDA;
            if (s == QS_OK) s = qs_sum_batched(b, probs, stream);
            if (s == QS_OK && cudaEventRecord(e1, st) != cudaSuccess) s = QS_ERR_CUDA;
            float ms = 0.0f;
            if (s == QS_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                s = QS_ERR_CUDA;
            if (s == QS_OK && ms < tb) tb = ms;
        }
        if (s == QS_OK && tb < best_ms) {
            best_ms = tb;
            best = tpt == 8 ? 0 : tpt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != QS_OK) {
        b->tpt_cap = keep;
        b->mode = keep_mode;
        return s == QS_ERR_CUDA ? bfail(QS_ERR_CUDA, "qs_batch_autotune: timing failed") : s;
    }
    b->mode = best == 0 ? QS_BATCH_CONCURRENT : QS_BATCH_PERSISTENT;
    b->tpt_cap = best == 0 ? keep : best;
    if (chosen) *chosen = best;
    return QS_OK;
}
