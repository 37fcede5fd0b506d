// Tensor-core projection for sm_103a (arXiv 2410.01316, Sec. 2.1 eq.
// kernel_sum_sliced; App. C Step 1):
//
//     U[p][n] = u_{n,p} = G tau <x_n, xi_p>,   D = X Xi_s^T on the tensor cores
//
// Two persistent kernels.  tc_project_persistent: one CTA per SM computes
// 128-point x 256-slice tiles; TMA streams K-major slabs of the points (A,
// 128 rows) and of the scaled directions (B, 256 rows) into 64-byte-swizzled
// shared memory through a ring of stages; one thread issues tcgen05.mma into
// one of two 256-column FP32 accumulators in tensor memory while eight warps
// read the other back with tcgen05.ld and store U with one coalesced 128-byte
// row segment per warp and slice.  tc_project_pair (the default): a cluster
// of two CTAs on an SM pair computes 256-point x 256-slice tiles with
// cta_group::2 MMAs (M = 256), each CTA holding half of every A and B slab;
// per SM that cuts the shared-memory traffic of a k-step from 160 to about
// 106 bytes per clock at the tensor pipe's rate, below the 128 the shared
// memory delivers, which bounded the single-SM form.
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
    static constexpr int ESZ = 2, BK = 32, NOPS = 2, KSTEP = 16;
    static constexpr uint32_t IDESC = make_idesc(1, TILE_M, TILE_N);
};
template <>
struct TcCfg<1> {  // TF32
    static constexpr int ESZ = 4, BK = 16, NOPS = 1, KSTEP = 8;
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


// ---------------------------------------------------------------------------
// Persistent form: one CTA per SM walks the tiles t = blockIdx.x, +gridDim.x,
// ... (slice tile fastest, so CTAs running together share point tiles in L2).
// Warp 0 lane 0 streams k-slabs through a STAGES-deep ring; warp 1 lane 0
// issues the MMAs into one of two 256-column TMEM accumulators; warps 2..9
// drain the other accumulator to U meanwhile (two warps per TMEM lane
// quarter), so a tile's epilogue overlaps the next tile's MMAs; with a short
// K (small d) the tile is bound by these stores of U.  Barriers: full/empty per ring stage, tfull/tempty
// per accumulator (tempty counts the epilogue warps).  Every wait is
// bounded; a role that gives up raises the shared abort flag and the error
// flag, and the others stop at their next tile.
// ---------------------------------------------------------------------------
template <int KIND>
struct PCfg;
template <>
struct PCfg<0> {  // BF16x3: 48 KB stages
    static constexpr int STAGES = 4;
};
template <>
struct PCfg<1> {  // TF32: 24 KB stages
    static constexpr int STAGES = 8;
};

template <int KIND>
__host__ __device__ constexpr int tcp_smem_bytes()
{
    return 1024 + PCfg<KIND>::STAGES * stage_bytes<KIND>() + 256;
}

constexpr int TCP_EPI_WARPS = 8;  // two per TMEM lane quarter, each storing half the columns
constexpr int TCP_THREADS = 32 * (2 + TCP_EPI_WARPS);

template <int KIND>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    tc_project_persistent(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                          const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, int d,
                          int P, int64_t n_base, int64_t N, float* __restrict__ U, int64_t ldU, unsigned int* flag)
{
    using C = TcCfg<KIND>;
    constexpr int ST = PCfg<KIND>::STAGES;
    constexpr int SB = stage_bytes<KIND>();
    extern __shared__ uint8_t smem_raw[];
    __shared__ volatile int abort_all;
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t tiles = (base + 1023u) & ~1023u;
    const uint32_t bars = tiles + ST * SB;
    const uint32_t full0 = bars;              // full[s]   = full0 + 8 s
    const uint32_t empty0 = bars + 8 * ST;    // empty[s]  = empty0 + 8 s
    const uint32_t tfull0 = bars + 16 * ST;   // tfull[a]  = tfull0 + 8 a
    const uint32_t tempty0 = tfull0 + 16;     // tempty[a] = tempty0 + 8 a
    const uint32_t drain = tempty0 + 16;      // all MMAs of the CTA have completed
    const uint32_t tmem_slot = drain + 8;
    uint32_t* tmem_slot_ptr = reinterpret_cast<uint32_t*>(smem_raw + (tmem_slot - base));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nkb = (d + C::BK - 1) / C::BK;
    const int ptiles = (P + TILE_N - 1) / TILE_N;
    const int64_t ntiles = (N + TILE_M - 1) / TILE_M;
    const int64_t T = ntiles * ptiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, TCP_EPI_WARPS);
        }
        mbar_init(drain, 1);
        abort_all = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                     "r"(2 * TILE_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot_ptr;

    if (warp == 0 && lane == 0) {
        // TMA producer: slab g of the CTA's sequence uses stage g % ST
        bool ok = true;
        int64_t g = 0;
        for (int64_t t = blockIdx.x; t < T && ok && !abort_all; t += gridDim.x) {
            const int p0 = (int)(t % ptiles) * TILE_N;
            const int n0 = (int)(n_base + (t / ptiles) * TILE_M);
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % ST);
                const uint32_t ph = (uint32_t)(g / ST) & 1u;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
                    ok = false;
                    break;
                }
                const uint32_t fb = full0 + 8 * s;
                const uint32_t st = tiles + s * SB;
                const int kc = kb * C::BK;
                mbar_expect_tx(fb, SB);
                tma_load_2d(st, &mA0, kc, n0, fb);
                if (C::NOPS == 2) tma_load_2d(st + A_BYTES, &mA1, kc, n0, fb);
                tma_load_2d(st + C::NOPS * A_BYTES, &mB0, kc, p0, fb);
                if (C::NOPS == 2) tma_load_2d(st + C::NOPS * A_BYTES + B_BYTES, &mB1, kc, p0, fb);
            }
        }
        // no copy of this CTA may still be in flight when it exits
        for (int64_t h = (g > ST ? g - ST : 0); h < g; ++h)
            if (!mbar_wait(full0 + 8 * (int)(h % ST), (uint32_t)(h / ST) & 1u)) ok = false;
        if (!ok) {
            abort_all = 1;
            atomicOr(flag, QS_FLAG_TIMEOUT);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        int64_t g = 0;
        int i = 0;
        for (int64_t t = blockIdx.x; t < T && ok && !abort_all; t += gridDim.x, ++i) {
            const int a = i & 1;
            if (!mbar_wait(tempty0 + 8 * a, (((uint32_t)i >> 1) & 1u) ^ 1u)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(a * TILE_N);
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % ST);
                if (!mbar_wait(full0 + 8 * s, (uint32_t)(g / ST) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = tiles + s * SB;
                const uint32_t a0 = st, a1 = st + A_BYTES;
                const uint32_t b0 = st + C::NOPS * A_BYTES, b1 = b0 + B_BYTES;
#pragma unroll
                for (int k = 0; k < C::BK / C::KSTEP; ++k) {
                    const uint32_t off = (uint32_t)(k * C::KSTEP * C::ESZ);
                    const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                    if (KIND == 0) {
                        mma_f16(dt, sw64_desc(a0 + off), sw64_desc(b0 + off), C::IDESC, acc);
                        mma_f16(dt, sw64_desc(a0 + off), sw64_desc(b1 + off), C::IDESC, 1u);
                        mma_f16(dt, sw64_desc(a1 + off), sw64_desc(b0 + off), C::IDESC, 1u);
                    } else {
                        mma_tf32(dt, sw64_desc(a0 + off), sw64_desc(b0 + off), C::IDESC, acc);
                    }
                }
                mma_commit(empty0 + 8 * s);
            }
            if (ok) mma_commit(tfull0 + 8 * a);  // arrives once the tile's MMAs have completed
        }
        // before the tensor memory is freed, every MMA issued above must have finished
        mma_commit(drain);
        if (!mbar_wait(drain, 0)) ok = false;
        if (!ok) {
            abort_all = 1;
            atomicOr(flag, QS_FLAG_TIMEOUT);
        }
    } else if (warp >= 2) {
        // epilogue: TMEM lane quarter q = warp % 4 holds points n0 + 32 q + lane;
        // the two warps of a quarter take columns [128 h, 128 h + 128)
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        int i = 0;
        for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++i) {
            if (abort_all) break;
            const int a = i & 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * a, ((uint32_t)i >> 1) & 1u));
            if (!got) {
                if (lane == 0) {
                    abort_all = 1;
                    atomicOr(flag, QS_FLAG_TIMEOUT);
                }
                break;
            }
            tc_fence_after();
            const int p0 = (int)(t % ptiles) * TILE_N;
            const int64_t n = n_base + (t / ptiles) * TILE_M + 32 * q + lane;
            const uint32_t trow = tmem + (uint32_t)(a * TILE_N) + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
            for (int c = h * (TILE_N / 2); c < (h + 1) * (TILE_N / 2); c += 32) {
                float v[32];
                __syncwarp();
                tmem_ld32(trow + (uint32_t)c, v);
                const int pc = p0 + c;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (pc + j < P) U[(size_t)(pc + j) * ldU + n] = v[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * a) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TILE_N)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// SM-pair form (cta_group::2): a cluster of two CTAs on an SM pair computes
// 256-point x 256-slice tiles with one M = 256 MMA per k-step.  CTA r of the
// pair (r = cluster rank) keeps points n0 + 128 r .. + 127 (A) and slices
// p0 + 128 r .. + 127 (B) of each k-slab in its own shared memory; the pair's
// MMA takes A from each CTA and B from both, so per SM a k-step reads half
// the B bytes of the single-SM form from shared memory and TMA writes two
// thirds of its bytes there.  The even CTA (the leader) issues the MMAs; its
// producer announces both CTAs' TMA bytes on its full barrier of the stage,
// on which the odd CTA's copies complete too (an mbarrier's transaction count
// may run below zero until the announcement); the leader's commits arrive on the empty, tfull and drain barriers of both
// CTAs (multicast); each CTA's tensor memory holds the accumulator rows of
// its own 128 points, drained to U by its eight epilogue warps, which arrive
// on the leader's tempty barriers.  One warp of each CTA allocates and frees
// the pair's tensor memory together.  Waits on barriers are bounded as in the
// single-SM form; both CTAs always reach the two closing cluster barriers.
// Teardown: the producers stop only at the end of their work or when their
// own bounded wait on an empty barrier runs out (never on the other warps'
// abort flag), so both normally issue the same number of stages; each
// publishes that count in the leader's shared memory before the first closing
// barrier.  The leader then completes any stage only one CTA issued (after a
// timeout: it announces the odd CTA's bytes, or issues its own copies of the
// stage a second time, which rewrites the same bytes, in place of the odd
// CTA's missing ones) and waits, bounded, for the last ring of stages on its
// full barriers, which count both CTAs' bytes.  Only then do the CTAs pass
// the second barrier and exit, so no copy is in flight into either CTA's
// shared memory when it exits unless that final bounded wait itself runs out.
// ---------------------------------------------------------------------------
template <int KIND>
struct PairCfg;
template <>
struct PairCfg<0> {  // BF16x3: 32 KB stages
    static constexpr int STAGES = 6;
};
template <>
struct PairCfg<1> {  // TF32: 16 KB stages
    static constexpr int STAGES = 12;
};

constexpr int PB_ROWS = TILE_N / 2;            // slices of a B slab held by one CTA
constexpr int PB_BYTES = PB_ROWS * ROW_BYTES;

template <int KIND>
__host__ __device__ constexpr int pair_stage_bytes()
{
    return TcCfg<KIND>::NOPS * (A_BYTES + PB_BYTES);
}

template <int KIND>
__host__ __device__ constexpr int pair_smem_bytes()
{
    return 1024 + PairCfg<KIND>::STAGES * pair_stage_bytes<KIND>() + 256;
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_count_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// All threads of both CTAs; release / acquire orders their shared-memory work.
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the variable at shared::cta address `addr` in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cl_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_bar) : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on a
// barrier of either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t cl_bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(cl_bar)
        : "memory");
}

__device__ __forceinline__ void mma_f16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive once on the barrier at offset `bar` of both CTAs of the pair when all
// MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((unsigned short)3)
        : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    tc_project_pair(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                    const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, int d, int P,
                    int64_t n_base, int64_t N, float* __restrict__ U, int64_t ldU, unsigned int* flag)
{
    using C = TcCfg<KIND>;
    constexpr int ST = PairCfg<KIND>::STAGES;
    constexpr int SB = pair_stage_bytes<KIND>();
    constexpr uint32_t IDESC = make_idesc(KIND == 0 ? 1u : 2u, 2 * TILE_M, TILE_N);
    constexpr int PAIR_M = 2 * TILE_M;
    extern __shared__ uint8_t smem_raw[];
    __shared__ volatile int abort_all;
    __shared__ long long issued[2];           // stages issued by each CTA's producer (the leader's copy is read)
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t tiles = (base + 1023u) & ~1023u;
    const uint32_t bars = tiles + ST * SB;
    const uint32_t full0 = bars;              // full[s]   = full0 + 8 s   (used in the leader)
    const uint32_t empty0 = bars + 8 * ST;    // empty[s]  = empty0 + 8 s
    const uint32_t tfull0 = bars + 16 * ST;   // tfull[a]  = tfull0 + 8 a
    const uint32_t tempty0 = tfull0 + 16;     // tempty[a] = tempty0 + 8 a (used in the leader)
    const uint32_t drain = tempty0 + 16;      // every MMA of the pair has completed
    const uint32_t tmem_slot = drain + 8;
    uint32_t* tmem_slot_ptr = reinterpret_cast<uint32_t*>(smem_raw + (tmem_slot - base));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int64_t cid = cluster_id_x();
    const int64_t ncl = cluster_count_x();
    const int nkb = (d + C::BK - 1) / C::BK;
    const int ptiles = (P + TILE_N - 1) / TILE_N;
    const int64_t ntiles = (N + PAIR_M - 1) / PAIR_M;
    const int64_t T = ntiles * ptiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(full0 + 8 * s, 1);  // the leader's producer
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 2 * TCP_EPI_WARPS);
        }
        mbar_init(drain, 1);
        abort_all = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                     "r"(2 * TILE_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *tmem_slot_ptr;

    // this CTA's copies of k-slab kb of tile t into stage s, completing on the
    // leader's full barrier of that stage
    auto issue_stage = [&](int64_t t, int kb, int s) {
        const int pr = (int)(t % ptiles) * TILE_N + (int)rank * PB_ROWS;
        const int nr = (int)(n_base + (t / ptiles) * PAIR_M + (int64_t)rank * TILE_M);
        const uint32_t fb = cluster_addr(full0 + 8 * s, 0);  // the leader's full[s]
        const uint32_t st = tiles + s * SB;
        const int kc = kb * C::BK;
        tma_load_2d_pair(st, &mA0, kc, nr, fb);
        if (C::NOPS == 2) tma_load_2d_pair(st + A_BYTES, &mA1, kc, nr, fb);
        tma_load_2d_pair(st + C::NOPS * A_BYTES, &mB0, kc, pr, fb);
        if (C::NOPS == 2) tma_load_2d_pair(st + C::NOPS * A_BYTES + PB_BYTES, &mB1, kc, pr, fb);
    };

    if (warp == 0 && lane == 0) {
        // TMA producer of this CTA's halves: slab g (tile step g / nkb, k-slab
        // g % nkb) uses stage g % ST.  It stops only at the end of its slabs
        // or when its own bounded wait runs out, so both CTAs' producers issue
        // the same stages unless one of them timed out (the teardown below
        // completes the difference)
        bool ok = true;
        int64_t g = 0;
        for (int64_t t = cid; t < T && ok; t += ncl) {
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = (int)(g % ST);
                const uint32_t ph = (uint32_t)(g / ST) & 1u;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
                    ok = false;
                    break;
                }
                if (leader) mbar_expect_tx(full0 + 8 * s, 2 * SB);
                issue_stage(t, kb, s);
            }
        }
        // publish the count in the leader's shared memory (ordered before the
        // first closing cluster barrier by its release)
        const uint32_t slot = cluster_addr(smem_u32(&issued[rank]), 0);
        asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(slot), "l"((long long)g) : "memory");
        if (!ok) {
            abort_all = 1;
            atomicOr(flag, QS_FLAG_TIMEOUT);
        }
    } else if (warp == 1 && lane == 0) {
        bool ok = true;
        if (leader) {
            // MMA issuer of the pair
            int64_t g = 0;
            int i = 0;
            for (int64_t t = cid; t < T && ok && !abort_all; t += ncl, ++i) {
                const int a = i & 1;
                if (!mbar_wait(tempty0 + 8 * a, (((uint32_t)i >> 1) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(a * TILE_N);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % ST);
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)(g / ST) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = tiles + s * SB;
                    const uint32_t a0 = st, a1 = st + A_BYTES;
                    const uint32_t b0 = st + C::NOPS * A_BYTES, b1 = b0 + PB_BYTES;
#pragma unroll
                    for (int k = 0; k < C::BK / C::KSTEP; ++k) {
                        const uint32_t off = (uint32_t)(k * C::KSTEP * C::ESZ);
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        if (KIND == 0) {
                            mma_f16_pair(dt, sw64_desc(a0 + off), sw64_desc(b0 + off), IDESC, acc);
                            mma_f16_pair(dt, sw64_desc(a0 + off), sw64_desc(b1 + off), IDESC, 1u);
                            mma_f16_pair(dt, sw64_desc(a1 + off), sw64_desc(b0 + off), IDESC, 1u);
                        } else {
                            mma_tf32_pair(dt, sw64_desc(a0 + off), sw64_desc(b0 + off), IDESC, acc);
                        }
                    }
                    mma_commit_pair(empty0 + 8 * s);
                }
                if (ok) mma_commit_pair(tfull0 + 8 * a);
            }
            mma_commit_pair(drain);
        }
        // tensor memory of both CTAs is written by the leader's MMAs: wait for all of them
        if (!mbar_wait(drain, 0)) ok = false;
        if (!ok) {
            abort_all = 1;
            atomicOr(flag, QS_FLAG_TIMEOUT);
        }
    } else if (warp >= 2) {
        // epilogue: lane quarter q = warp % 4 of this CTA's accumulator holds
        // points nr + 32 q + lane; the two warps of a quarter split the columns
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t tempty_l[2] = {cluster_addr(tempty0, 0), cluster_addr(tempty0 + 8, 0)};
        int i = 0;
        for (int64_t t = cid; t < T; t += ncl, ++i) {
            if (abort_all) break;
            const int a = i & 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * a, ((uint32_t)i >> 1) & 1u));
            if (!got) {
                if (lane == 0) {
                    abort_all = 1;
                    atomicOr(flag, QS_FLAG_TIMEOUT);
                }
                break;
            }
            tc_fence_after();
            const int p0 = (int)(t % ptiles) * TILE_N;
            const int64_t n = n_base + (t / ptiles) * PAIR_M + (int64_t)rank * TILE_M + 32 * q + lane;
            // a 256-row pair tile can pass the 128-rounded width of U: store rows < n_base + N only
            const bool row_ok = n < n_base + N;
            const uint32_t trow = tmem + (uint32_t)(a * TILE_N) + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
            for (int c = h * (TILE_N / 2); c < (h + 1) * (TILE_N / 2); c += 32) {
                float v[32];
                __syncwarp();
                tmem_ld32(trow + (uint32_t)c, v);
                const int pc = p0 + c;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (row_ok && pc + j < P) U[(size_t)(pc + j) * ldU + n] = v[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(tempty_l[a]);
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // both producers' counts are in the leader's shared memory
    if (leader && warp == 0 && lane == 0) {
        // every copy of the pair completes on the leader's full barriers; a
        // stage's phase completes once both CTAs' bytes have landed.  Stages
        // below max(g0, g1) - ST completed before the last ring was issued
        // (a stage is issued only after the MMAs consumed the one ST slabs
        // earlier), and |g0 - g1| <= ST for the same reason.
        const int64_t g0 = issued[0], g1 = issued[1];
        const int64_t hi = g0 > g1 ? g0 : g1, mid = g0 > g1 ? g1 : g0;
        bool ok = true;
        for (int64_t h = mid; h < hi; ++h) {
            if (g0 > g1) issue_stage(cid + (h / nkb) * ncl, (int)(h % nkb), (int)(h % ST));  // the odd CTA's bytes
                                                                                           // will not come: send ours again
            else mbar_expect_tx(full0 + 8 * (int)(h % ST), SB);  // announce the odd CTA's bytes
        }
        for (int64_t h = (hi > ST ? hi - ST : 0); h < hi; ++h)
            if (!mbar_wait(full0 + 8 * (int)(h % ST), (uint32_t)(h / ST) & 1u)) ok = false;
        if (!ok) atomicOr(flag, QS_FLAG_TIMEOUT);
    }
    __syncthreads();
    cluster_sync_all();  // no copy of the pair is in flight; both CTAs are done with its barriers and tensor memory
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TILE_N)
                     : "memory");
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

cudaError_t qs_launch_split_bf16(const float* X, int64_t rows, int d, int ldk, void* hi, void* lo, cudaStream_t st,
                                 int max_blocks)
{
    if (rows <= 0) return cudaSuccess;
    const int64_t total = rows * (int64_t)(ldk / 4);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (vec)
        split_bf16_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, (__nv_bfloat16*)hi,
                                                                   (__nv_bfloat16*)lo);
    else
        split_bf16_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, (__nv_bfloat16*)hi,
                                                                    (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t qs_launch_round_tf32(const float* X, int64_t rows, int d, int ldk, float* out, cudaStream_t st,
                                 int max_blocks)
{
    if (rows <= 0) return cudaSuccess;
    const int64_t total = rows * (int64_t)ldk;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    round_tf32_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, rows, d, ldk, out);
    return cudaGetLastError();
}

namespace {

// Co-resident clusters of the SM-pair kernel (0 if it cannot run here).
template <int KIND>
int pair_clusters()
{
    static int n = -1;
    if (n < 0) {
        int v = 0;
        const int smem = pair_smem_bytes<KIND>();
        if (cudaFuncSetAttribute(tc_project_pair<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(2, 1, 1);
            cfg.blockDim = dim3(TCP_THREADS, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&v, tc_project_pair<KIND>, &cfg) != cudaSuccess) v = 0;
        }
        cudaGetLastError();  // a refusal here only means the pair form is unavailable
        n = v;
    }
    return n;
}

template <int KIND>
cudaError_t launch_pair(const CUtensorMap* m, int64_t n_base, int64_t N, int d, int P, float* U, int64_t ldU,
                        unsigned int* flag, cudaStream_t st)
{
    const int ncl_max = pair_clusters<KIND>();
    if (ncl_max <= 0) return cudaErrorNotSupported;
    const int smem = pair_smem_bytes<KIND>();
    const int64_t T = ((N + 2 * TILE_M - 1) / (2 * TILE_M)) * ((P + TILE_N - 1) / TILE_N);
    const int ncl = (int)(T < ncl_max ? T : ncl_max);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
    cfg.blockDim = dim3(TCP_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // maps 4 / 5: the directions with 128-row boxes (one CTA's half of a B slab)
    const CUtensorMap& a1 = KIND == 0 ? m[1] : m[0];
    const CUtensorMap& b1 = KIND == 0 ? m[5] : m[4];
    cudaError_t e = cudaLaunchKernelEx(&cfg, tc_project_pair<KIND>, m[0], a1, m[4], b1, d, P, n_base, N, U, ldU, flag);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

bool qs_tc_pair_available(int kind)
{
    return (kind == 0 ? pair_clusters<0>() : pair_clusters<1>()) > 0;
}

int qs_tc_pair_ctas(int kind)
{
    return 2 * (kind == 0 ? pair_clusters<0>() : pair_clusters<1>());
}

// maps: [A0, A1, B0, B1, B0 half, B1 half] (A1 / B1 unused by TF32), each a
// 64-byte-aligned CUtensorMap; B maps 2 / 3 have 256-row boxes, 4 / 5 128-row boxes.
cudaError_t qs_launch_project_tc(int kind, const void* maps, int64_t n_base, int64_t N, int d, int P, float* U,
                                 int64_t ldU, unsigned int* flag, cudaStream_t st, bool pair)
{
    if (N <= 0) return cudaSuccess;
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps);
    if (pair) return kind == 0 ? launch_pair<0>(m, n_base, N, d, P, U, ldU, flag, st)
                               : launch_pair<1>(m, n_base, N, d, P, U, ldU, flag, st);
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int64_t T = ((N + TILE_M - 1) / TILE_M) * ((P + TILE_N - 1) / TILE_N);
    const unsigned grid = (unsigned)(T < sms ? T : sms);
    if (kind == 0) {
        const int smem = tcp_smem_bytes<0>();
        cudaError_t e =
            cudaFuncSetAttribute(tc_project_persistent<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        tc_project_persistent<0><<<grid, TCP_THREADS, smem, st>>>(m[0], m[1], m[2], m[3], d, P, n_base, N, U, ldU, flag);
    } else {
        const int smem = tcp_smem_bytes<1>();
        cudaError_t e =
            cudaFuncSetAttribute(tc_project_persistent<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        tc_project_persistent<1><<<grid, TCP_THREADS, smem, st>>>(m[0], m[0], m[2], m[2], d, P, n_base, N, U, ldU, flag);
    }
    return cudaGetLastError();
}
