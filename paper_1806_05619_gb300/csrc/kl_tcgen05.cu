// KL field synthesis on the 5th-generation tensor cores (sm_103a).
//
// For one grid level the truncated KL expansion (eq. truncatedKL) of every
// sample is a dense contraction
//     Z[p][b] = sum_m Psi[p][m] * C[b][m],  Psi[p][m] = psi_{a_m}(x1_p) psi_{b_m}(x2_p),
//                                          C[b][m]   = sqrt(theta_m) y_{b,m},
// p over the level's cells, b over the samples, m over the s modes; the
// coefficient is k = exp(Z). Tiles of 128 cells x NT samples: TMA brings
// 128-byte-swizzled K blocks of Psi (A operand, K-major) and C (B operand,
// K-major) into shared memory through an mbarrier ring; one thread issues
// tcgen05.mma kind::tf32 into an FP32 accumulator in TMEM; eight epilogue
// warps (two per 32-lane quarter of TMEM, half of the tile's samples each)
// read their TMEM lanes (one cell each) with tcgen05.ld, apply exp and
// store k sample by sample, coalesced across cells. The CTAs are persistent
// and warp-specialised with two TMEM accumulators, so that the epilogue of
// one tile runs while the tensor cores work on the next.
// Operands are rounded to TF32 (round to nearest) when they are built.
//
// Split-BF16 variant: every operand x is split into hi = bf16(x) and
// lo = bf16(x - hi), and the contraction sums the three products hi*hi,
// hi*lo and lo*hi (the lo*lo term is below FP32 resolution of the sum). The
// three products are one GEMM over a tripled K: Psi rows hold [hi | hi | lo],
// C rows [hi | lo | hi], so the kernel is the TF32 one with kind::f16 MMAs on
// BF16 operands; a 128-byte K block holds 64 BF16 instead of 32 TF32.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

#include "kl_tcgen05.h"

namespace {

constexpr int kTileM = 128;      // cells per CTA (TMEM lanes)
constexpr int kKBlock = 32;      // K elements per stage (128 bytes of FP32)
// shared-memory ring stages: 192 KB of A (128 cells) and B (NT samples) K blocks
template <int NT>
constexpr int stages_for()
{
    return NT == 128 ? 6 : 4;
}
constexpr uint32_t kErrTimeout = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with `parity` to complete, giving up after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 255u) == 0 && now_ns() - t0 > 1000000000ull) break;
    }
    atomicOr(err, static_cast<int>(kErrTimeout));
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
    d |= static_cast<uint64_t>(1) << 16;                   // leading byte offset (unused for this layout)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;           // stride byte offset: next 8-row atom
    d |= static_cast<uint64_t>(1) << 46;                   // descriptor version
    d |= static_cast<uint64_t>(2) << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Instruction descriptor: kind::f16 with A = B = BF16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

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
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Wait for the phase with `parity`; gives up when another role of the CTA has
// given up (*abort set) or after about a second (then sets *abort and the
// timeout bit of *err), so that every role leaves its loops.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort, int* err)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort) return false;
            if (now_ns() - t0 > 1000000000ull) break;
        }
    }
    *abort = 1;
    atomicOr(err, static_cast<int>(kErrTimeout));
    return false;
}

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kEpiWarps = 8;                       // two per TMEM lane quarter, half the columns each
constexpr int kTcThreads = 64 + 32 * kEpiWarps;    // TMA warp, MMA warp, epilogue warps

// Persistent CTAs (one per SM) walk the 128-cell x NT-sample tiles of the
// level, sample tiles fastest (consecutive tiles share their Psi rows in L2).
// Warp 0 (one thread) streams the K blocks of Psi and C of every tile through
// the shared-memory ring; warp 1 (one thread) issues the MMAs of a tile into
// one of two TMEM accumulators (2 x NT columns) and commits; warps 2-9 read
// the other accumulator (warp w owns TMEM lanes 32 (w % 4) .. and half of the
// columns), apply exp and store, so the epilogue of tile i overlaps the MMAs
// of tile i + 1 and the ring never drains between tiles. The ring holds 192 KB
// of K blocks: four stages of 128 + 256 rows, six of 128 + 128 (one and a half
// tiles at s = 100).
template <int NT, bool BF>
__global__ void __launch_bounds__(kTcThreads, 1) kl_tc_kernel(const __grid_constant__ CUtensorMap tm_psi,
                                                              const __grid_constant__ CUtensorMap tm_c, int M, int B,
                                                              int nk, float* __restrict__ kout, size_t kstride,
                                                              int* err)
{
    constexpr int kStages = stages_for<NT>();
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned stage buffers (the 128-byte swizzle atom)
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr uint32_t kABytes = kTileM * kKBlock * 4;
    constexpr uint32_t kBBytes = NT * kKBlock * 4;
    unsigned char* sa = smem;
    unsigned char* sb = smem + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sb + kStages * kBBytes);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;   // accumulator a holds a finished tile
    uint64_t* tempty = tfull + 2;        // accumulator a has been read out
    uint64_t* drained = tempty + 2;      // every MMA issued so far has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int ntiles = (B + NT - 1) / NT;
    const int tiles = ((M + kTileM - 1) / kTileM) * ntiles;  // the Psi map holds whole 128-row tiles (zero rows past M)

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpiWarps);
        }
        mbar_init(drained, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(static_cast<uint32_t>(2 * NT))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: K blocks of Psi rows m0.. and C rows b0.. of every tile
            uint32_t g = 0, issued = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
                const int m0 = (tile / ntiles) * kTileM, b0 = (tile % ntiles) * NT;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % kStages;
                    if (g >= kStages && !(ok = wait_or_abort(&empty[s], ((g / kStages) - 1) & 1, abort, err))) break;
                    mbar_expect_tx(&full[s], kABytes + kBBytes);
                    constexpr int kElems = BF ? 64 : kKBlock;  // elements per 128-byte K block
                    tma_load_2d(sa + s * kABytes, &tm_psi, &full[s], kb * kElems, m0);
                    tma_load_2d(sb + s * kBBytes, &tm_c, &full[s], kb * kElems, b0);
                    issued = g + 1;
                }
            }
            // let every copy this thread issued land before the CTA can leave
            for (uint32_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
                mbar_wait(&full[k % kStages], (k / kStages) & 1, err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile lt accumulates into columns (lt & 1) * NT
            constexpr uint32_t idesc = BF ? idesc_bf16(kTileM, NT) : idesc_tf32(kTileM, NT);
            uint32_t g = 0;
            bool ok = true;
            int lt = 0;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++lt) {
                const int a = lt & 1;
                if (lt >= 2 && !(ok = wait_or_abort(&tempty[a], ((lt >> 1) - 1) & 1, abort, err))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + static_cast<uint32_t>(a * NT);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const uint32_t s = g % kStages;
                    if (!(ok = wait_or_abort(&full[s], (g / kStages) & 1, abort, err))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ad = sdesc_sw128(smem_u32(sa + s * kABytes));
                    const uint64_t bd = sdesc_sw128(smem_u32(sb + s * kBBytes));
#pragma unroll
                    for (int k = 0; k < kKBlock / 8; ++k) {  // 32 bytes of K per MMA: 8 TF32 or 16 BF16
                        if constexpr (BF) mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
                        else mma_tf32(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&tfull[a]);
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(drained);
            mbar_wait(drained, 0, err);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 q .. 32 q + 31, q = w % 4 (cells m0 + 32 q + lane),
        // accumulator columns [h NT / 2, (h + 1) NT / 2), h = (w - 2) / 4
        const int q = warp & 3;
        const int c_lo = ((warp - 2) >> 2) * (NT / 2);
        int lt = 0;
        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++lt) {
            const int a = lt & 1;
            // warp-uniform: the TMEM loads below are .sync.aligned
            const bool ready = __all_sync(0xffffffffu, wait_or_abort(&tfull[a], (lt >> 1) & 1, abort, err) ? 1 : 0);
            if (!ready) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / ntiles) * kTileM, b0 = (tile % ntiles) * NT;
            const int p = m0 + q * 32 + lane;
#pragma unroll 1
            for (int c = c_lo; c < c_lo + NT / 2; c += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(a * NT + c), v);
                if (p < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int b = b0 + c + j;
                        if (b < B) kout[static_cast<size_t>(b) * kstride + p] = __expf(v[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive1(&tempty[a]);
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(static_cast<uint32_t>(2 * NT))
                     : "memory");
    }
}

__device__ __forceinline__ float to_tf32(double v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(static_cast<float>(v)));
    return __uint_as_float(r);
}

// Psi[p][m] = tf32(psi_{a_m}(x1) psi_{b_m}(x2)) for p = i2*n + i1, zero for m >= s.
__global__ void kl_build_psi(const double* __restrict__ psi1d, int n, int s, int kpad, const int* __restrict__ ma,
                             const int* __restrict__ mb, float* __restrict__ out)
{
    const int64_t total = static_cast<int64_t>(n) * n * kpad;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx % kpad);
        const int64_t p = idx / kpad;
        const int i2 = static_cast<int>(p / n), i1 = static_cast<int>(p % n);
        out[idx] = m < s ? to_tf32(psi1d[static_cast<size_t>(ma[m]) * n + i1] * psi1d[static_cast<size_t>(mb[m]) * n + i2])
                         : 0.0f;
    }
}

// C[i][m] = tf32(sqrt(theta_m) y_{canon_i, m}), zero for m >= s.
__global__ void kl_build_c(const double* __restrict__ Y, const int* __restrict__ canon, int count, int s, int kpad,
                           const double* __restrict__ sqrt_theta, float* __restrict__ out)
{
    const int64_t total = static_cast<int64_t>(count) * kpad;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx % kpad);
        const int i = static_cast<int>(idx / kpad);
        const size_t row = canon ? static_cast<size_t>(canon[i]) : static_cast<size_t>(i);
        out[idx] = m < s ? to_tf32(sqrt_theta[m] * Y[row * s + m]) : 0.0f;
    }
}

// hi + lo split of x (round to nearest both times)
__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    const float x = static_cast<float>(v);
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Psi3[p][j], j < 3 kp: [hi | hi | lo] of psi_{a_m}(x1) psi_{b_m}(x2), zero for m >= s.
__global__ void kl_build_psi_bf16x3(const double* __restrict__ psi1d, int n, int s, int kp, const int* __restrict__ ma,
                                    const int* __restrict__ mb, __nv_bfloat16* __restrict__ out)
{
    const int64_t total = static_cast<int64_t>(n) * n * kp;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx % kp);
        const int64_t p = idx / kp;
        const int i2 = static_cast<int>(p / n), i1 = static_cast<int>(p % n);
        __nv_bfloat16 hi = __float2bfloat16_rn(0.0f), lo = hi;
        if (m < s) split_bf16(psi1d[static_cast<size_t>(ma[m]) * n + i1] * psi1d[static_cast<size_t>(mb[m]) * n + i2], hi, lo);
        __nv_bfloat16* row = out + p * 3 * kp;
        row[m] = hi;
        row[kp + m] = hi;
        row[2 * kp + m] = lo;
    }
}

// Psi operand from dense FP64 modes (Matern, Nystrom): src[p * s + m] -> TF32
// row p, or the [hi | hi | lo] split rows; zero for m >= s.
__global__ void kl_build_psi_dense(const double* __restrict__ src, int64_t M, int s, int kp, int split,
                                   void* __restrict__ out)
{
    const int64_t total = M * kp;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx % kp);
        const int64_t p = idx / kp;
        const double v = m < s ? src[p * s + m] : 0.0;
        if (!split) {
            static_cast<float*>(out)[idx] = m < s ? to_tf32(v) : 0.0f;
        } else {
            __nv_bfloat16 hi = __float2bfloat16_rn(0.0f), lo = hi;
            if (m < s) split_bf16(v, hi, lo);
            __nv_bfloat16* row = static_cast<__nv_bfloat16*>(out) + p * 3 * kp;
            row[m] = hi;
            row[kp + m] = hi;
            row[2 * kp + m] = lo;
        }
    }
}

// C3[i][j]: [hi | lo | hi] of sqrt(theta_m) y_{canon_i, m}, zero for m >= s.
__global__ void kl_build_c_bf16x3(const double* __restrict__ Y, const int* __restrict__ canon, int count, int s, int kp,
                                  const double* __restrict__ sqrt_theta, __nv_bfloat16* __restrict__ out)
{
    const int64_t total = static_cast<int64_t>(count) * kp;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(idx % kp);
        const int i = static_cast<int>(idx / kp);
        const size_t src = canon ? static_cast<size_t>(canon[i]) : static_cast<size_t>(i);
        __nv_bfloat16 hi = __float2bfloat16_rn(0.0f), lo = hi;
        if (m < s) split_bf16(sqrt_theta[m] * Y[src * s + m], hi, lo);
        __nv_bfloat16* row = out + static_cast<size_t>(i) * 3 * kp;
        row[m] = hi;
        row[kp + m] = lo;
        row[2 * kp + m] = hi;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

// 2D map over rows x kdim (inner) elements of 4 (FP32) or 2 (BF16) bytes:
// box of one 128-byte K block x box_rows, 128-byte swizzle.
bool encode_2d(CUtensorMap* map, const void* base, uint64_t rows, uint64_t kdim, uint32_t box_rows, bool bf16)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const uint64_t es = bf16 ? 2 : 4;
    const cuuint64_t dims[2] = {kdim, rows};
    const cuuint64_t strides[1] = {kdim * es};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / es), box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kNT = 256;

size_t tc_smem_bytes(int nt = kNT)
{
    const int st = nt == 128 ? stages_for<128>() : stages_for<kNT>();
    return 1024 + st * (kTileM * kKBlock * 4 + static_cast<size_t>(nt) * kKBlock * 4) + (2 * st + 5) * 8 + 16;
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

namespace mlqmc_kl {

int kpad_for(int s)
{
    return (s + kKBlock - 1) / kKBlock * kKBlock;
}

int kdim_for(Variant v, int s)
{
    if (v == Variant::TF32) return kpad_for(s);
    return 3 * ((s + 63) / 64 * 64);  // three BF16 parts, each whole 64-element (128-byte) blocks
}

size_t row_bytes(Variant v, int s)
{
    return static_cast<size_t>(kdim_for(v, s)) * (v == Variant::TF32 ? 4 : 2);
}

bool build_psi_dense(Variant v, const double* d_modes, int64_t M, int s, void* d_out, cudaStream_t st)
{
    const int kp = v == Variant::TF32 ? kpad_for(s) : kdim_for(v, s) / 3;
    const int64_t total = M * kp;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 64)));
    kl_build_psi_dense<<<grid, 256, 0, st>>>(d_modes, M, s, kp, v == Variant::TF32 ? 0 : 1, d_out);
    return cudaGetLastError() == cudaSuccess;
}

bool build_psi(Variant v, const double* d_psi1d, int n, int s, const int* d_ma, const int* d_mb, void* d_out,
               cudaStream_t st)
{
    const int kp = v == Variant::TF32 ? kpad_for(s) : kdim_for(v, s) / 3;
    const int64_t total = static_cast<int64_t>(n) * n * kp;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 64));
    if (v == Variant::TF32) kl_build_psi<<<grid, 256, 0, st>>>(d_psi1d, n, s, kp, d_ma, d_mb, static_cast<float*>(d_out));
    else kl_build_psi_bf16x3<<<grid, 256, 0, st>>>(d_psi1d, n, s, kp, d_ma, d_mb, static_cast<__nv_bfloat16*>(d_out));
    return cudaGetLastError() == cudaSuccess;
}

bool build_c(Variant v, const double* d_Y, const int* d_canon, int count, int s, const double* d_sqrt_theta,
             void* d_out, cudaStream_t st)
{
    const int kp = v == Variant::TF32 ? kpad_for(s) : kdim_for(v, s) / 3;
    const int64_t total = static_cast<int64_t>(count) * kp;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 64)));
    if (v == Variant::TF32)
        kl_build_c<<<grid, 256, 0, st>>>(d_Y, d_canon, count, s, kp, d_sqrt_theta, static_cast<float*>(d_out));
    else
        kl_build_c_bf16x3<<<grid, 256, 0, st>>>(d_Y, d_canon, count, s, kp, d_sqrt_theta,
                                                static_cast<__nv_bfloat16*>(d_out));
    return cudaGetLastError() == cudaSuccess;
}

bool make_maps(Variant v, const void* d_psi, int M, const void* d_c, int rows_c, int s, TensorMaps* maps)
{
    const int kd = kdim_for(v, s);
    const bool bf = v == Variant::BF16X3;
    static_assert(sizeof(TensorMaps::psi) >= sizeof(CUtensorMap), "map storage");
    return encode_2d(reinterpret_cast<CUtensorMap*>(maps->psi), d_psi, static_cast<uint64_t>(M), kd, kTileM, bf) &&
           encode_2d(reinterpret_cast<CUtensorMap*>(maps->c), d_c, static_cast<uint64_t>(rows_c), kd, kNT, bf) &&
           encode_2d(reinterpret_cast<CUtensorMap*>(maps->c128), d_c, static_cast<uint64_t>(rows_c), kd, 128, bf);
}

bool prepare_kernel()
{
    const int b = static_cast<int>(tc_smem_bytes(kNT)), b128 = static_cast<int>(tc_smem_bytes(128));
    return cudaFuncSetAttribute(kl_tc_kernel<kNT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kl_tc_kernel<kNT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kl_tc_kernel<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b128) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kl_tc_kernel<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b128) ==
               cudaSuccess;
}

bool launch(Variant v, const TensorMaps& maps, int M, int B, int s, float* d_k, size_t kstride, int* d_err,
            cudaStream_t st, int nt)
{
    if (M <= 0 || B <= 0 || (nt != 128 && nt != kNT)) return false;
    const int nk = static_cast<int>(row_bytes(v, s) / 128);  // 128-byte K blocks
    CUtensorMap tp, tc;
    std::memcpy(&tp, maps.psi, sizeof(CUtensorMap));
    std::memcpy(&tc, nt == 128 ? maps.c128 : maps.c, sizeof(CUtensorMap));
    const int tiles = ((M + kTileM - 1) / kTileM) * ((B + nt - 1) / nt);
    const int grid = std::min(tiles, sm_count());  // persistent: one CTA per SM
    const size_t smem = tc_smem_bytes(nt);
    if (nt == 128) {
        if (v == Variant::TF32) kl_tc_kernel<128, false><<<grid, kTcThreads, smem, st>>>(tp, tc, M, B, nk, d_k, kstride, d_err);
        else kl_tc_kernel<128, true><<<grid, kTcThreads, smem, st>>>(tp, tc, M, B, nk, d_k, kstride, d_err);
    } else {
        if (v == Variant::TF32) kl_tc_kernel<kNT, false><<<grid, kTcThreads, smem, st>>>(tp, tc, M, B, nk, d_k, kstride, d_err);
        else kl_tc_kernel<kNT, true><<<grid, kTcThreads, smem, st>>>(tp, tc, M, B, nk, d_k, kstride, d_err);
    }
    return cudaGetLastError() == cudaSuccess;
}

int tile_samples() { return kNT; }

}  // namespace mlqmc_kl
