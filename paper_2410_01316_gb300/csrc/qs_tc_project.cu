// Tensor-core projection for sm_103a (arXiv 2410.01316, Sec. 2.1 eq.
// kernel_sum_sliced; App. C Step 1):
//
//     U[p][n] = u_{n,p} = G tau <x_n, xi_p>,   D = X Xi_s^T on the tensor cores
//
// One CTA computes a 128-point x 256-slice tile.  TMA streams K-major tiles
// of the points (A, 128 rows) and of the scaled directions (B, 256 rows) into
// 64-byte-swizzled shared memory (64-byte k-slabs, two stages, 97 KB per CTA,
// so two CTAs share an SM and one's epilogue overlaps the other's MMAs); one
// thread issues tcgen05.mma with the FP32 accumulator in tensor memory (256
// columns); all four warps read the accumulator back with tcgen05.ld and store
// U with one coalesced 128-byte row segment per warp and slice.
//
// Two precision forms:
//   BF16x3  x = x_hi + x_lo and xi = xi_hi + xi_lo in BF16 (round to nearest);
//           D accumulates x_hi xi_hi + x_hi xi_lo + x_lo xi_hi  (kind::f16)
//   TF32    x and xi rounded to TF32 (round to nearest); one product (kind::tf32)
//
// Every mbarrier wait is bounded; on exhaustion the kernel sets the timeout
// bit of the plan's error flag, skips the remaining work and still frees its
// tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "qs_internal.cuh"

namespace {

constexpr int TILE_M = 128;             // points per tile (TMEM lanes)
constexpr int TILE_N = 256;             // slices per tile (TMEM columns)
constexpr uint32_t SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false once the spin limit is spent.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand tile in the
// 64-byte swizzle layout written by TMA: rows of 64 bytes, groups of 8 rows
// 512 bytes apart (stride byte offset), descriptor version 1, layout 4.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format `fmt` (BF16 = 1 for
// kind::f16, TF32 = 2 for kind::tf32), both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns; thread i receives lane (base + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int KIND>
struct TcCfg;
template <>
struct TcCfg<0> {  // BF16x3
    static constexpr int ESZ = 2, BK = 32, STAGES = 2, NOPS = 2, KSTEP = 16;
    static constexpr uint32_t IDESC = make_idesc(1, TILE_M, TILE_N);
};
template <>
struct TcCfg<1> {  // TF32
    static constexpr int ESZ = 4, BK = 16, STAGES = 4, NOPS = 1, KSTEP = 8;
    static constexpr uint32_t IDESC = make_idesc(2, TILE_M, TILE_N);
};

constexpr int ROW_BYTES = 64;               // one 64-byte swizzle row per operand row and k-slab
constexpr int A_BYTES = TILE_M * ROW_BYTES;
constexpr int B_BYTES = TILE_N * ROW_BYTES;

template <int KIND>
__host__ __device__ constexpr int stage_bytes()
{
    return TcCfg<KIND>::NOPS * (A_BYTES + B_BYTES);
}

template <int KIND>
__host__ __device__ constexpr int tc_smem_bytes()
{
    return 1024 + TcCfg<KIND>::STAGES * stage_bytes<KIND>() + 256;
}

// mA0/mA1: points (hi/lo for BF16x3), mB0/mB1: scaled directions.
template <int KIND>
__global__ void __launch_bounds__(128, 2)
    tc_project_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                      const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, int d,
                      int P, float* __restrict__ U, int64_t ldU, unsigned int* flag)
{
    using C = TcCfg<KIND>;
    constexpr int SB = stage_bytes<KIND>();
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t tiles = (base + 1023u) & ~1023u;
    const uint32_t bars = tiles + C::STAGES * SB;
    const uint32_t full0 = bars;                       // full[s]  = full0 + 8 s
    const uint32_t empty0 = bars + 8 * C::STAGES;      // empty[s] = empty0 + 8 s
    const uint32_t done = bars + 16 * C::STAGES;
    const uint32_t tmem_slot = done + 8;
    uint32_t* tmem_slot_ptr = reinterpret_cast<uint32_t*>(smem_raw + (tmem_slot - base));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int p0 = blockIdx.x * TILE_N;
    const int n0 = blockIdx.y * TILE_M;
    const int nkb = (d + C::BK - 1) / C::BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                     "r"(TILE_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot_ptr;

    if (warp == 0 && lane == 0) {
        // TMA producer
        bool ok = true;
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % C::STAGES;
            const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
                ok = false;
                break;
            }
            const uint32_t full = full0 + 8 * s;
            const uint32_t st = tiles + s * SB;
            const int kc = kb * C::BK;
            mbar_expect_tx(full, SB);
            tma_load_2d(st, &mA0, kc, n0, full);
            if (C::NOPS == 2) tma_load_2d(st + A_BYTES, &mA1, kc, n0, full);
            tma_load_2d(st + C::NOPS * A_BYTES, &mB0, kc, p0, full);
            if (C::NOPS == 2) tma_load_2d(st + C::NOPS * A_BYTES + B_BYTES, &mB1, kc, p0, full);
            issued = kb + 1;
        }
        // make sure no copy of this CTA is still in flight when it exits
        for (int kb = (issued > C::STAGES ? issued - C::STAGES : 0); kb < issued; ++kb)
            if (!mbar_wait(full0 + 8 * (kb % C::STAGES), (uint32_t)(kb / C::STAGES) & 1u)) ok = false;
        if (!ok) atomicOr(flag, QS_FLAG_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % C::STAGES;
            const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
            if (!mbar_wait(full0 + 8 * s, ph)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = tiles + s * SB;
            const uint32_t a0 = st, a1 = st + A_BYTES;
            const uint32_t b0 = st + C::NOPS * A_BYTES, b1 = b0 + B_BYTES;
#pragma unroll
            for (int k = 0; k < C::BK / C::KSTEP; ++k) {
                const uint32_t off = (uint32_t)(k * C::KSTEP * C::ESZ);  // 32 bytes per step
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                if (KIND == 0) {
                    mma_f16(tmem, sw64_desc(a0 + off), sw64_desc(b0 + off), C::IDESC, acc);
                    mma_f16(tmem, sw64_desc(a0 + off), sw64_desc(b1 + off), C::IDESC, 1u);
                    mma_f16(tmem, sw64_desc(a1 + off), sw64_desc(b0 + off), C::IDESC, 1u);
                } else {
                    mma_tf32(tmem, sw64_desc(a0 + off), sw64_desc(b0 + off), C::IDESC, acc);
                }
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);  // arrives once every MMA issued above has completed
        if (!ok) atomicOr(flag, QS_FLAG_TIMEOUT);
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes 32w..32w+31 = points n0 + 32w + lane.
    // Lanes leave the wait loop independently; the vote reconverges the warp
    // before the warp-collective tcgen05.ld.
    const bool got = __all_sync(0xffffffffu, mbar_wait(done, 0));
    tc_fence_after();
    if (got) {
        const int64_t n = (int64_t)n0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int c = 0; c < TILE_N; c += 32) {
            float v[32];
            __syncwarp();
            tmem_ld32(trow + (uint32_t)c, v);
            const int pc = p0 + c;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (pc + j < P) U[(size_t)(pc + j) * ldU + n] = v[j];
        }
    } else if (lane == 0) {
        atomicOr(flag, QS_FLAG_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TILE_N) : "memory");
    }
}

// BF16 split of an FP32 row-major matrix (rows x d) into hi and lo parts with
// row stride ldk (padding columns zero): hi = bf16_rn(v), lo = bf16_rn(v - hi).
// Each thread converts 4 consecutive entries of a row (ldk is a multiple of
// 8): one 16-byte load when the row has them (d % 4 == 0 and aligned), one
// 8-byte store per output.
__device__ __forceinline__ void split4(float4 v, uint2& h, uint2& l)
{
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f01 = __bfloat1622float2(h01);
    const float2 f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
    h = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    l = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
}

template <bool VEC>
__global__ void split_bf16_kernel(const float* __restrict__ X, int64_t rows, int d, int ldk,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo)
{
    const int g4 = ldk >> 2;
    const int64_t total = rows * (int64_t)g4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / g4;
        const int k = (int)(i - r * g4) << 2;
        float4 v;
        if (VEC && k + 3 < d) {
            v = __ldg(reinterpret_cast<const float4*>(X + r * d + k));
        } else {
            v.x = k < d ? __ldg(&X[r * d + k]) : 0.0f;
            v.y = k + 1 < d ? __ldg(&X[r * d + k + 1]) : 0.0f;
            v.z = k + 2 < d ? __ldg(&X[r * d + k + 2]) : 0.0f;
            v.w = k + 3 < d ? __ldg(&X[r * d + k + 3]) : 0.0f;
        }
        uint2 h, l;
        split4(v, h, l);
        *reinterpret_cast<uint2*>(hi + r * ldk + k) = h;
        *reinterpret_cast<uint2*>(lo + r * ldk + k) = l;
    }
}

// Round an FP32 row-major matrix (rows x d) to TF32 (nearest, ties away) with
// row stride ldk (padding columns zero).
__global__ void round_tf32_kernel(const float* __restrict__ X, int64_t rows, int d, int ldk, float* __restrict__ out)
{
    const int64_t total = rows * (int64_t)ldk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ldk;
        const int k = (int)(i - r * ldk);
        const float v = k < d ? __ldg(&X[r * d + k]) : 0.0f;
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
        out[i] = __uint_as_float(t);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

// 2-D K-major tensor map: `rows` rows of `d` elements with a row stride of
// ldk elements; box = one 64-byte swizzle row (BK elements) x box_rows rows.
// Coordinates past d or rows read zeros.
bool qs_make_tmap(void* map_out, const void* base, int elem_bytes, int d, int64_t rows, int ldk, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)ldk * (cuuint64_t)elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1, 1};
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(map_out), dt, 2, const_cast<void*>(base), gdim, gstride, box,
                     estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t qs_launch_split_bf16(const float* X, int64_t rows, int d, int ldk, void* hi, void* lo, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const int64_t total = rows * (int64_t)(ldk / 4);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (vec)
        split_bf16_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, (__nv_bfloat16*)hi,
                                                                   (__nv_bfloat16*)lo);
    else
        split_bf16_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, (__nv_bfloat16*)hi,
                                                                    (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t qs_launch_round_tf32(const float* X, int64_t rows, int d, int ldk, float* out, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    const int64_t total = rows * (int64_t)ldk;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    round_tf32_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, out);
    return cudaGetLastError();
}

// maps: [A0, A1, B0, B1] (A1 / B1 unused by TF32), each a 64-byte-aligned CUtensorMap.
cudaError_t qs_launch_project_tc(int kind, const void* maps, int64_t N, int d, int P, float* U, int64_t ldU,
                                 unsigned int* flag, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps);
    dim3 grid((unsigned)((P + TILE_N - 1) / TILE_N), (unsigned)((N + TILE_M - 1) / TILE_M));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    if (kind == 0) {
        const int smem = tc_smem_bytes<0>();
        cudaError_t e = cudaFuncSetAttribute(tc_project_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        tc_project_kernel<0><<<grid, 128, smem, st>>>(m[0], m[1], m[2], m[3], d, P, U, ldU, flag);
    } else {
        const int smem = tc_smem_bytes<1>();
        cudaError_t e = cudaFuncSetAttribute(tc_project_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        tc_project_kernel<1><<<grid, 128, smem, st>>>(m[0], m[0], m[2], m[2], d, P, U, ldU, flag);
    }
    return cudaGetLastError();
}
