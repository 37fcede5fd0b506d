// Device helpers shared by the grid kernels: the shared-memory real FFT and
// filter of a slice grid, and the cp.async staging of filtered rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsdev {

// ---------------------------------------------------------------------------
// In-place radix-2 complex FFT of length n = G/2 in shared memory.
// Forward uses e^{-2 pi i j / len}, inverse e^{+...}; both unnormalised.
// tw[t] = e^{-2 pi i t / G}, t < G/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool INV>
__device__ inline void fft_inplace(float2* z, int n, int log2n, const float2* __restrict__ tw, int G)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int j = (int)(__brev((unsigned)i) >> (32 - log2n));
        if (j > i) {
            const float2 t = z[i];
            z[i] = z[j];
            z[j] = t;
        }
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        const int stride = G / len;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int pos = b & (half - 1);
            const int i = ((b - pos) << 1) + pos;
            const int j = i + half;
            float2 wv = __ldg(&tw[pos * stride]);
            if (INV) wv.y = -wv.y;
            const float2 a = z[i];
            const float2 t = cmul(z[j], wv);
            z[i] = make_float2(a.x + t.x, a.y + t.y);
            z[j] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
}

// Real-input FFT post-processing, filter by D, and pre-processing of the
// real-output inverse, all on the packed spectrum z (length Gh = G/2):
//   z_j = g_{2j} + i g_{2j+1},  Z = FFT_Gh(z)
//   X_k = (Z_k + conj Z_{Gh-k})/2 + e^{-2 pi i k/G} (Z_k - conj Z_{Gh-k})/(2i)   (k = 0..Gh)
//   Y_k = D_k X_k
//   Z'_k = (Y_k + conj Y_{Gh-k}) + i e^{2 pi i k/G} (Y_k - conj Y_{Gh-k})       (k < Gh)
// so that IFFT_Gh(Z') interleaves the real sequence h_l = sum_k Y_k e^{2 pi i k l/G}.
// DERIV: the filter is i g_k with the real table g (derivative coefficients
// 2 pi i k c_k over psi^2), i.e. Y_k = i g_k X_k.
template <bool DERIV>
__device__ inline void real_filter(float2* z, int Gh, const float* __restrict__ D, const float2* __restrict__ tw)
{
    for (int k = threadIdx.x; k <= (Gh >> 1); k += blockDim.x) {
        if (k == 0) {
            const float2 z0 = z[0];
            if (DERIV) {
                // g_0 = 0 and g_{Gh} = 0 (Gh > N_ft/2): the real parts at k = 0, Gh vanish
                z[0] = make_float2(0.0f, 0.0f);
                continue;
            }
            const float y0 = __ldg(&D[0]) * (z0.x + z0.y);
            const float yh = __ldg(&D[Gh]) * (z0.x - z0.y);
            z[0] = make_float2(y0 + yh, y0 - yh);
            continue;
        }
        const int k2 = Gh - k;
        const float2 zk = z[k];
        const float2 zc = make_float2(z[k2].x, -z[k2].y);  // conj Z_{Gh-k}
        const float2 A = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 B = make_float2(0.5f * (zk.y - zc.y), -0.5f * (zk.x - zc.x));  // -i (Zk - Zc)/2
        const float2 t = __ldg(&tw[k]);
        const float2 tB = cmul(t, B);
        const float2 Xk = make_float2(A.x + tB.x, A.y + tB.y);
        const float2 Xk2 = make_float2(A.x - tB.x, -(A.y - tB.y));  // conj(A - t B)
        const float dk = __ldg(&D[k]);
        const float dk2 = __ldg(&D[k2]);
        const float2 Yk = DERIV ? make_float2(-dk * Xk.y, dk * Xk.x) : make_float2(dk * Xk.x, dk * Xk.y);
        const float2 Yk2 = DERIV ? make_float2(-dk2 * Xk2.y, dk2 * Xk2.x) : make_float2(dk2 * Xk2.x, dk2 * Xk2.y);
        const float2 tc = make_float2(t.x, -t.y);  // e^{+2 pi i k / G}
        // Z'_k = (Yk + conj Yk2) + i tc (Yk - conj Yk2)
        {
            const float2 sum = make_float2(Yk.x + Yk2.x, Yk.y - Yk2.y);
            const float2 dif = make_float2(Yk.x - Yk2.x, Yk.y + Yk2.y);
            const float2 r = cmul(tc, dif);
            z[k] = make_float2(sum.x - r.y, sum.y + r.x);
        }
        // Z'_{k2} = (Yk2 + conj Yk) + i (-t) (Yk2 - conj Yk)
        {
            const float2 sum = make_float2(Yk2.x + Yk.x, Yk2.y - Yk.y);
            const float2 dif = make_float2(Yk2.x - Yk.x, Yk2.y + Yk.y);
            const float2 r = cmul(make_float2(-t.x, -t.y), dif);
            z[k2] = make_float2(sum.x - r.y, sum.y + r.x);
        }
    }
}

constexpr int IT_THREADS = 256;
constexpr int ROW_PAD = 16;  // >= QS_MAX_W, keeps rows 64-byte aligned

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copy the G-cell row `src` into `dst` followed by its first ROW_PAD cells.
__device__ __forceinline__ void stage_row(float* dst, const float* src, int G)
{
    const int n16 = (G + ROW_PAD) >> 2;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
        const int c = (i << 2) < G ? (i << 2) : (i << 2) - G;
        cp_async16(dst + (i << 2), src + c);
    }
    cp_async_commit();
}


// ---------------------------------------------------------------------------
// One 128-slice x 128-point tile of the FP32 projection GEMM
//     U[p][n] = sum_j A[p][j] X[n][j]   (A = G tau Xi, X points, both K-major)
// by a CTA of 256 threads: 8-deep k slabs double-buffered in shared memory
// (`smem`: 2 x 8 x 256 floats = 16 KB), 8 x 8 outputs per thread.  Rows
// p >= P are not stored; columns n0..n0+127 are stored (U needs ldU >=
// round_up(N, 128)).
// ---------------------------------------------------------------------------
constexpr int GT_BM = 128;
constexpr int GT_BN = 128;
constexpr int GT_BK = 8;

template <bool VEC>
__device__ __forceinline__ void gemm_load_slab(const float* __restrict__ A, int P, const float* __restrict__ X,
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
__device__ inline void gemm_tile_fp32(const float* __restrict__ X, int64_t N, int d, const float* __restrict__ A,
                                      int P, float* __restrict__ U, int64_t ldU, int p0, int64_t n0, float* smem)
{
    float(*As)[GT_BK][GT_BM] = reinterpret_cast<float(*)[GT_BK][GT_BM]>(smem);
    float(*Bs)[GT_BK][GT_BN] = reinterpret_cast<float(*)[GT_BK][GT_BN]>(smem + 2 * GT_BK * GT_BM);
    const int tid = threadIdx.x;
    const int tx = tid & 15;
    const int ty = tid >> 4;
    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    float ra[4], rb[4];
    const int nk = (d + GT_BK - 1) / GT_BK;
    gemm_load_slab<VEC>(A, P, X, N, d, p0, n0, 0, lrow, lk, ra, rb);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        As[0][lk + i][lrow] = ra[i];
        Bs[0][lk + i][lrow] = rb[i];
    }
    __syncthreads();

    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) gemm_load_slab<VEC>(A, P, X, N, d, p0, n0, (kt + 1) * GT_BK, lrow, lk, ra, rb);
#pragma unroll
        for (int k = 0; k < GT_BK; ++k) {
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

}  // namespace qsdev
