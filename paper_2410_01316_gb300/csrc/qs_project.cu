// Projection step of the sliced sum (arXiv 2410.01316, Sec. 2.1 eq.
// kernel_sum_sliced and App. C Step 1): for every slice p and point n,
//
//     U[p][n] = u_{n,p} = G tau <x_n, xi_p>
//
// i.e. the GEMM U = Xi_s X^T with Xi_s = (G tau) Xi (P x d) and X (N x d),
// both row-major with d contiguous.  This file holds the plain FP32 SIMT form:
// 128 x 128 output tiles, 8-deep k slabs double-buffered in shared memory,
// 8 x 8 outputs per thread.
#include "qs_internal.cuh"

namespace {

constexpr int BM = 128;  // slices per tile
constexpr int BN = 128;  // points per tile
constexpr int BK = 8;    // reduction slab

template <bool VEC>
__device__ __forceinline__ void load_slab(const float* __restrict__ A, int P, const float* __restrict__ X,
                                          int64_t N, int d, int p0, int64_t n0, int k0, int lrow, int lk,
                                          float (&ra)[4], float (&rb)[4])
{
    const int gp = p0 + lrow;
    const int64_t gn = n0 + lrow;
    const int kk = k0 + lk;
    if (VEC && kk + 3 < d) {
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
        if (gp < P) va = __ldg(reinterpret_cast<const float4*>(A + (size_t)gp * d + kk));
        if (gn < N) vb = __ldg(reinterpret_cast<const float4*>(X + (size_t)gn * d + kk));
        ra[0] = va.x; ra[1] = va.y; ra[2] = va.z; ra[3] = va.w;
        rb[0] = vb.x; rb[1] = vb.y; rb[2] = vb.z; rb[3] = vb.w;
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ra[i] = (gp < P && kk + i < d) ? __ldg(A + (size_t)gp * d + kk + i) : 0.0f;
            rb[i] = (gn < N && kk + i < d) ? __ldg(X + (size_t)gn * d + kk + i) : 0.0f;
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(256) project_fp32_kernel(const float* __restrict__ X, int64_t N, int d,
                                                           const float* __restrict__ A, int P,
                                                           float* __restrict__ U, int64_t ldU)
{
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15;
    const int ty = tid >> 4;
    // blockIdx.x walks the slice tiles so that CTAs sharing one X tile run
    // back to back and X is read from DRAM once
    const int p0 = blockIdx.x * BM;
    const int64_t n0 = (int64_t)blockIdx.y * BN;
    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    float ra[4], rb[4];
    const int nk = (d + BK - 1) / BK;
    load_slab<VEC>(A, P, X, N, d, p0, n0, 0, lrow, lk, ra, rb);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        As[0][lk + i][lrow] = ra[i];
        Bs[0][lk + i][lrow] = rb[i];
    }
    __syncthreads();

    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load_slab<VEC>(A, P, X, N, d, p0, n0, (kt + 1) * BK, lrow, lk, ra, rb);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
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
        if (kt + 1 < nk) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                As[cur ^ 1][lk + i][lrow] = ra[i];
                Bs[cur ^ 1][lk + i][lrow] = rb[i];
            }
        }
        __syncthreads();
    }

    // rows: p0 + ty*4 + i (i < 4) and p0 + 64 + ty*4 + (i - 4); columns likewise
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int p = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (p >= P) continue;
        float* row = U + (size_t)p * ldU + n0;
        *reinterpret_cast<float4*>(row + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(row + 64 + tx * 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
}

}  // namespace

// U must have ldU >= round_up(N, 128) columns and ldU % 4 == 0 (the tile
// stores whole 128-column blocks; columns >= N receive zeros).
cudaError_t qs_launch_project_fp32(const float* X, int64_t N, int d, const float* xi_s, int P, float* U,
                                   int64_t ldU, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((N + BN - 1) / BN));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(xi_s) & 15) == 0);
    if (vec)
        project_fp32_kernel<true><<<grid, 256, 0, st>>>(X, N, d, xi_s, P, U, ldU);
    else
        project_fp32_kernel<false><<<grid, 256, 0, st>>>(X, N, d, xi_s, P, U, ldU);
    return cudaGetLastError();
}
