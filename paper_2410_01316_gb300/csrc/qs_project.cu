// Projection step of the sliced sum (arXiv 2410.01316, Sec. 2.1 eq.
// kernel_sum_sliced and App. C Step 1): for every slice p and point n,
//
//     U[p][n] = u_{n,p} = G tau <x_n, xi_p>
//
// i.e. the GEMM U = Xi_s X^T with Xi_s = (G tau) Xi (P x d) and X (N x d),
// both row-major with d contiguous.  This file holds the plain FP32 SIMT form
// (the tile routine gemm_tile_fp32 is shared with the batched kernel).
#include "qs_device.cuh"
#include "qs_internal.cuh"

using namespace qsdev;

namespace {

template <bool VEC>
__global__ void __launch_bounds__(256) project_fp32_kernel(const float* __restrict__ X, int64_t N, int d,
                                                           const float* __restrict__ A, int P,
                                                           float* __restrict__ U, int64_t ldU)
{
    __shared__ __align__(16) float smem[4 * GT_BK * GT_BM];
    // blockIdx.x walks the slice tiles so that CTAs sharing one X tile run
    // back to back and X is read from DRAM once
    gemm_tile_fp32<VEC>(X, N, d, A, P, U, ldU, blockIdx.x * GT_BM, (int64_t)blockIdx.y * GT_BN, smem);
}

}  // namespace

// U must have ldU >= round_up(N, 128) columns and ldU % 4 == 0 (the tile
// stores whole 128-column blocks; columns >= N receive zeros).
cudaError_t qs_launch_project_fp32(const float* X, int64_t N, int d, const float* xi_s, int P, float* U,
                                   int64_t ldU, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((P + GT_BM - 1) / GT_BM), (unsigned)((N + GT_BN - 1) / GT_BN));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(xi_s) & 15) == 0);
    if (vec)
        project_fp32_kernel<true><<<grid, 256, 0, st>>>(X, N, d, xi_s, P, U, ldU);
    else
        project_fp32_kernel<false><<<grid, 256, 0, st>>>(X, N, d, xi_s, P, U, ldU);
    return cudaGetLastError();
}
