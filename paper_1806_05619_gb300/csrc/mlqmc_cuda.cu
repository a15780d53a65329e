// CUDA path of the MG-MLQMC library (sm_103a).
//
// One call of mlqmc_sample_levels runs SampleAndSolve (Algorithm 1) for a list
// of samples. Samples are ranked by finest level, descending; every level t
// keeps a pool with one block of arrays per sample whose FMG reaches t
// (B_t samples, B_t non-increasing in t), so sample i uses block i at every
// level. All grid work is level-synchronous: each kb_* kernel is one flat grid
// over the B_t samples of one level (KL field, faces, red-black sweeps,
// residual/restriction, prolongation, FP64 refinement steps, QoI), so samples
// of uneven finest levels share every launch of the levels they have in
// common (Sec. 4 FMG, Fig. FMG). Only level 0 is per sample: kb_level0 factors
// the banded level-0 matrix (one warp per sample) and kb_coarse does the
// coarse solves of the V-cycles (one thread per sample). k_sums then forms the
// reuse sums (eq. Upsilon-reuse) in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "fmg_device.cuh"
#include "mlqmc_internal.h"
#include "rbgs_stream.h"
#include "rbgs_tma.h"
#include "resid_tma.h"
#include "ptx_async.cuh"
#include "rbgs_whole.h"
#include "matern_nystrom.h"

using namespace mlqmc_dev;

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products, key bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Coordinate j's 64 bits of the block (j/2, c1, c2, tag) under key `seed`.
__device__ __forceinline__ uint64_t philox_coord(uint32_t c1, uint32_t c2, uint32_t tag, uint64_t seed, int j)
{
    const uint4 o = philox10(make_uint4(static_cast<uint32_t>(j) >> 1, c1, c2, tag), static_cast<uint32_t>(seed),
                             static_cast<uint32_t>(seed >> 32));
    return (j & 1) ? ((static_cast<uint64_t>(o.w) << 32) | o.z) : ((static_cast<uint64_t>(o.y) << 32) | o.x);
}

// Point bits of sample (level, r, n), coordinate j: lattice sequence in
// radical-inverse order plus a 64-bit random shift (mod 2^64), or MC bits.
__device__ __forceinline__ uint64_t point_bits(int sampler, uint64_t seed, const uint32_t* z, int level, int r,
                                               int64_t n, int j)
{
    if (sampler == MLQMC_SAMPLER_LATTICE) {
        const uint32_t t = __brev(static_cast<uint32_t>(n)) * z[j];
        const uint64_t shift = philox_coord(static_cast<uint32_t>(r), static_cast<uint32_t>(level), 0x53484654u, seed, j);
        return (static_cast<uint64_t>(t) << 32) + shift;
    }
    return philox_coord(static_cast<uint32_t>(n), (static_cast<uint32_t>(r) << 8) | static_cast<uint32_t>(level),
                        0x4D43524Eu, seed, j);
}

// The lattice shifts depend only on (level, r, j): a table of them, filled
// once per context by philox_coord itself, replaces the ten Philox rounds
// per point of the batched point kernels (same bits).
__global__ void k_shift_table(int R, int L, int s, uint64_t seed, uint64_t* __restrict__ tab)
{
    const int64_t total = static_cast<int64_t>(R) * L * s;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(idx % s);
        const int64_t rest = idx / s;
        const int r = static_cast<int>(rest % R), level = static_cast<int>(rest / R);
        tab[idx] = philox_coord(static_cast<uint32_t>(r), static_cast<uint32_t>(level), 0x53484654u, seed, j);
    }
}

// point_bits, with the lattice shift from the table when there is one
__device__ __forceinline__ uint64_t point_bits_tab(int sampler, uint64_t seed, const uint32_t* z,
                                                   const uint64_t* tab, int R, int s, int level, int r, int64_t n,
                                                   int j)
{
    if (tab && sampler == MLQMC_SAMPLER_LATTICE) {
        const uint32_t t = __brev(static_cast<uint32_t>(n)) * z[j];
        return (static_cast<uint64_t>(t) << 32) + tab[(static_cast<size_t>(level) * R + r) * s + j];
    }
    return point_bits(sampler, seed, z, level, r, n, j);
}

// Points and normals y = Phi^-1(u) (Sec. 3.2). fp32 (mixed forms, whose
// normals only enter FP32 and tensor-core arithmetic): Phi^-1 in FP32, each
// half of (0, 1) taken from its own end (1 - u formed exactly in integers),
// so both tails keep float resolution; the FP64 form uses FP64.
__global__ void k_points(const SampleDesc* __restrict__ smp, int count, int s, int sampler, uint64_t seed,
                         const uint32_t* __restrict__ z, const uint64_t* __restrict__ tab, int R,
                         double* __restrict__ Y, uint64_t* __restrict__ bits, int fp32)
{
    const int64_t total = static_cast<int64_t>(count) * s;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(idx / s);
        const int j = static_cast<int>(idx - static_cast<int64_t>(q) * s);
        const SampleDesc d = smp[q];
        const uint64_t x = point_bits_tab(sampler, seed, z, tab, R, s, d.level, d.r, d.n, j);
        const size_t o = static_cast<size_t>(d.canon) * s + j;
        if (bits) bits[o] = x;
        if (Y && fp32) {
            const uint64_t k = x >> 11;  // u = (k + 1/2) 2^-53
            const bool lo = k < (1ull << 52);
            const uint64_t kk = lo ? k : ((1ull << 53) - 1ull) - k;  // 1 - u = (kk + 1/2) 2^-53 in the upper half
            const float y = normcdfinvf(fmaf(__ull2float_rn(kk), 0x1p-53f, 0x1p-54f));
            Y[o] = widen(lo ? y : -y);
        } else if (Y) {
            const double u = (static_cast<double>(x >> 11) + 0.5) * 0x1.0p-53;  // open (0,1)
            Y[o] = normcdfinv(u);
        }
    }
}

// Mixed TF32 form with separable modes: the chunk's normals (the FP32
// inverse CDF of k_points, stored widened in Y) and, from the same FP64
// product sqrt(theta_m) y_m, its FP32 rounding (the coefficients of the SIMT
// synthesis, as k_coef32) and its TF32 rounding (the tensor-core C operand,
// zero-padded to kpad columns, as kl_build_c), in one pass over (sample,
// column): the three kernels' values without re-reading Y. Samples in rank
// order with canon = rank (the batched calls). Y and c32 may be null (every
// level's field from the tensor cores: only C is read).
__global__ void k_points_mixed(const SampleDesc* __restrict__ smp, int count, int s, int kpad, FastDiv by_kpad,
                               int sampler, uint64_t seed, const uint32_t* __restrict__ z,
                               const uint64_t* __restrict__ tab, int R, const double* __restrict__ sq,
                               double* __restrict__ Y, float* __restrict__ c32, float* __restrict__ C)
{
    const uint32_t total = static_cast<uint32_t>(count) * static_cast<uint32_t>(kpad);
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int i = static_cast<int>(by_kpad.div(idx));
        const int m = static_cast<int>(idx - static_cast<uint32_t>(i) * static_cast<uint32_t>(kpad));
        if (m >= s) {
            C[idx] = 0.0f;
            continue;
        }
        const SampleDesc d = smp[i];
        const uint64_t x = point_bits_tab(sampler, seed, z, tab, R, s, d.level, d.r, d.n, m);
        const uint64_t k = x >> 11;  // u = (k + 1/2) 2^-53
        const bool lo = k < (1ull << 52);
        const uint64_t kk = lo ? k : ((1ull << 53) - 1ull) - k;
        const float y = normcdfinvf(fmaf(__ull2float_rn(kk), 0x1p-53f, 0x1p-54f));
        const double yw = widen(lo ? y : -y);
        if (Y) Y[static_cast<size_t>(d.canon) * s + m] = yw;
        const float pf = narrow(sq[m] * yw);
        if (c32) c32[static_cast<size_t>(i) * s + m] = pf;
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(pf));
        C[idx] = __uint_as_float(r);
    }
}

// Flat loops in 32-bit indices: chunks are cut so that every level's
// samples x elements stays below 2^31 (see mlqmc_sample_levels).
#define GRID_STRIDE(idx, total)                                                                       \
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < static_cast<uint32_t>(total); \
         idx += gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// Level 0, one thread per sample. GB300 issues FP64 at a few operations per
// clock per SM, charged per warp instruction whatever the active lanes, so
// the per-sample band work runs with every lane busy on its own sample.
// Band factor of h0^2 A_0 (bandwidth n0): entry (r, d) = L(r, r-d) of sample i
// at fac[(r*(n0+1) + d) * stride + i] (coalesced across samples); the
// diagonal d = 0 holds 1/L(r, r).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T band_a(const T* kx, const T* ky, int n0, int r, int l)
{
    const int r1 = r % n0, r2 = r / n0;
    if (l == 1 && r1 > 0) return -kx[r2 * kx_pitch(n0) + r1];
    if (l == n0) return -ky[r2 * n0 + r1];
    return T(0);
}

// Factor, exact FP64 solve with f = 1, F_0; the mixed forms also keep an FP32
// copy of the factor for the coarse solves of their FP32 V-cycles.
template <typename T, bool MX>
__global__ void kb_level0(FmgArgs A, int B)
{
    const int n0 = A.n0, N = n0 * n0, W = n0 + 1;
    const size_t cs = A.chol.stride;
    double* fac = reinterpret_cast<double*>(A.chol.base);
    GRID_STRIDE(ii, B)
    {
        const int i = static_cast<int>(ii);
        const Lv<T> L0 = view<T>(A, 0, i);
        for (int j = 0; j < N; ++j) {
            const int j1 = j % n0, j2 = j / n0;
            double d = widen(L0.kx[j2 * kx_pitch(n0) + j1]) + widen(L0.kx[j2 * kx_pitch(n0) + j1 + 1]) +
                       widen(L0.ky[j2 * n0 + j1]) + widen(L0.ky[(j2 + 1) * n0 + j1]);
            for (int q = 1; q <= n0 && q <= j; ++q) {
                const double l = fac[static_cast<size_t>(j * W + q) * cs + i];
                d -= l * l;
            }
            const double rl = rsqrt64(d);
            fac[static_cast<size_t>(j * W) * cs + i] = rl;
            for (int l = 1; l <= n0 && j + l < N; ++l) {
                const int r = j + l;
                double a = widen(band_a(L0.kx, L0.ky, n0, r, l));
                for (int tt = (r - n0 > 0 ? r - n0 : 0); tt < j; ++tt)
                    a -= fac[static_cast<size_t>(r * W + (r - tt)) * cs + i] * fac[static_cast<size_t>(j * W + (j - tt)) * cs + i];
                fac[static_cast<size_t>(r * W + l) * cs + i] = a * rl;
            }
        }
        // exact solution of level 0 with f = 1 (the first node of Fig. FMG)
        double* x = (MX || A.refine) ? L0.u64 : reinterpret_cast<double*>(L0.u);
        const double h2 = 1.0 / (static_cast<double>(n0) * n0);
        for (int r = 0; r < N; ++r) {
            double v = h2;
            for (int q = 1; q <= n0 && q <= r; ++q) v -= fac[static_cast<size_t>(r * W + q) * cs + i] * x[r - q];
            x[r] = v * fac[static_cast<size_t>(r * W) * cs + i];
        }
        for (int r = N - 1; r >= 0; --r) {
            double v = x[r];
            for (int q = 1; q <= n0 && r + q < N; ++q) v -= fac[static_cast<size_t>((r + q) * W + q) * cs + i] * x[r + q];
            x[r] = v * fac[static_cast<size_t>(r * W) * cs + i];
        }
        double F0;
        if (A.qoi == MLQMC_QOI_MEAN) {
            double acc = 0.0;
            for (int r = 0; r < N; ++r) acc += x[r];
            F0 = acc / static_cast<double>(N);
        } else {
            const int m = n0 / 2;
            F0 = 0.25 * (x[(m - 1) * n0 + (m - 1)] + x[(m - 1) * n0 + m] + x[m * n0 + (m - 1)] + x[m * n0 + m]);
        }
        A.F[static_cast<size_t>(i) * A.n_levels] = F0;
        if constexpr (MX) {
            float* u32 = reinterpret_cast<float*>(L0.u);  // FP32 copy for the first FMG interpolation
            for (int r = 0; r < N; ++r) u32[r] = static_cast<float>(x[r]);
            float* f32 = reinterpret_cast<float*>(A.chol32);
            for (int q = 0; q < N * W; ++q) f32[static_cast<size_t>(q) * cs + i] = static_cast<float>(fac[static_cast<size_t>(q) * cs + i]);
        }
    }
}

// Coarse solve of the V-cycles, u_0 = A_0^{-1} bc_0, one thread per sample, in
// the working precision. SM: the thread's vector lives in shared memory
// (element r at xs[r * blockDim + tid]), else in its pool block.
template <typename T, bool SM>
__global__ void kb_coarse(FmgArgs A, int B)
{
    extern __shared__ unsigned char sraw[];
    const int n0 = A.n0, N = n0 * n0, W = n0 + 1;
    const T h2 = T(1) / (T(n0) * T(n0));
    const T* fac = reinterpret_cast<const T*>(sizeof(T) == 4 ? A.chol32 : A.chol.base);
    const size_t cs = A.chol.stride;
    const int bd = blockDim.x;
    for (int64_t ii = blockIdx.x * static_cast<int64_t>(bd) + threadIdx.x;; ii += static_cast<int64_t>(gridDim.x) * bd) {
        if (ii >= B) break;
        const int i = static_cast<int>(ii);
        if (A.active && !A.active[i]) continue;
        const T* b = at<T>(A.lv[0].bc, i);
        T* xo = at<T>(A.lv[0].u, i);
        T* xs = SM ? reinterpret_cast<T*>(sraw) + threadIdx.x : xo;
        const int xst = SM ? bd : 1;
        for (int r = 0; r < N; ++r) {
            T v = h2 * b[r];
            for (int q = 1; q <= n0 && q <= r; ++q) v -= fac[static_cast<size_t>(r * W + q) * cs + i] * xs[(r - q) * xst];
            xs[r * xst] = v * fac[static_cast<size_t>(r * W) * cs + i];
        }
        for (int r = N - 1; r >= 0; --r) {
            T v = xs[r * xst];
            for (int q = 1; q <= n0 && r + q < N; ++q) v -= fac[static_cast<size_t>((r + q) * W + q) * cs + i] * xs[(r + q) * xst];
            xs[r * xst] = v * fac[static_cast<size_t>(r * W) * cs + i];
        }
        if (SM)
            for (int r = 0; r < N; ++r) xo[r] = xs[r * xst];
    }
}

// Level 0 for n0 = NC fixed at compile time, one thread per sample, with the
// working rows of the factorisation in shared memory: column j of L needs
// rows j..j+NC only, so a ring of NC+1 rows per thread (transposed by thread:
// conflict-free) holds them; a finished row goes to the global factor once.
// The forward substitution runs along with the factorisation, its last NC
// values in registers and every value stored into the sample's solution
// array, which the backward substitution then overwrites in place (again
// with the last NC values in registers); shared memory holds the ring only,
// so that all samples of a call fit on the GPU at once. Same arithmetic, in
// the same order, as kb_level0.
template <typename T, bool MX, int NC>
__global__ void __launch_bounds__(64) kb_level0_fixed(FmgArgs A, int B)
{
    constexpr int N = NC * NC, W = NC + 1, TPB = 64;
    extern __shared__ double l0sh[];
    double* ring = l0sh;  // [(slot * W + e) * TPB + tid]
    const int tid = threadIdx.x;
    const size_t cs = A.chol.stride;
    double* fac = reinterpret_cast<double*>(A.chol.base);
    float* f32 = reinterpret_cast<float*>(A.chol32);
    const double h2 = 1.0 / (static_cast<double>(NC) * NC);
    for (int base = blockIdx.x * TPB; base < B; base += gridDim.x * TPB) {
        const int i = base + tid;
        if (i >= B) continue;  // no barriers in this kernel: shared rows are private to the thread
        auto Rs = [&](int slot, int e) -> double& { return ring[(slot * W + e) * TPB + tid]; };
        const Lv<T> L0 = view<T>(A, 0, i);
        double* x = (MX || A.refine) ? L0.u64 : reinterpret_cast<double*>(L0.u);
        double win[NC];  // win[q - 1] = y_(j - q), the forward values of the last NC rows
#pragma unroll
        for (int q = 0; q < NC; ++q) win[q] = 0.0;
        // step j: row j's diagonal, its forward-substitution value, the row to
        // global memory, then column j of L for rows j+1..j+NC (ring slot of
        // row r: r mod W; FULL: j >= NC, every loop has its whole, compile-time range)
        auto step = [&](int j, auto full) {
            constexpr bool FULL = decltype(full)::value;
            const int s0 = j % W;
            auto slot = [&](int l) { return s0 + l >= W ? s0 + l - W : s0 + l; };  // slot of row j + l
            const int j1 = j % NC, j2 = j / NC;
            double d = widen(L0.kx[j2 * kx_pitch(NC) + j1]) + widen(L0.kx[j2 * kx_pitch(NC) + j1 + 1]) +
                       widen(L0.ky[j2 * NC + j1]) + widen(L0.ky[(j2 + 1) * NC + j1]);
#pragma unroll
            for (int q = 1; q <= NC; ++q) {
                if (!FULL && q > j) break;
                const double l = Rs(s0, q);
                d -= l * l;
            }
            const double rl = rsqrt64(d);
            Rs(s0, 0) = rl;
            double v = h2;  // forward substitution, f = 1
#pragma unroll
            for (int q = 1; q <= NC; ++q) {
                if (!FULL && q > j) break;
                v -= Rs(s0, q) * win[q - 1];
            }
            const double yj = v * rl;
            x[j] = yj;
#pragma unroll
            for (int q = NC - 1; q > 0; --q) win[q] = win[q - 1];
            win[0] = yj;
#pragma unroll
            for (int e = 0; e <= NC; ++e) {
                if (!FULL && e > j) break;
                fac[static_cast<size_t>(j * W + e) * cs + i] = Rs(s0, e);
                if constexpr (MX) f32[static_cast<size_t>(j * W + e) * cs + i] = narrow(Rs(s0, e));
            }
#pragma unroll
            for (int l = 1; l <= NC; ++l) {
                const int r = j + l;
                if (r >= N) break;
                double a = widen(band_a(L0.kx, L0.ky, NC, r, l));
                const int sr = slot(l);
                if constexpr (FULL) {
#pragma unroll
                    for (int u = 0; u < NC - l; ++u) {  // tt = r - NC + u = j - (NC - l) + u
                        a -= Rs(sr, NC - u) * Rs(s0, NC - l - u);
                    }
                } else {
                    for (int tt = (r - NC > 0 ? r - NC : 0); tt < j; ++tt) a -= Rs(sr, r - tt) * Rs(s0, j - tt);
                }
                Rs(sr, l) = a * rl;
            }
        };
        for (int j = 0; j < NC; ++j) step(j, std::false_type());
        for (int j = NC; j < N; ++j) step(j, std::true_type());
        // backward: x_r = (y_r - sum_q L(r+q, r) x_(r+q)) / L(r, r), win[q - 1] = x_(r+q)
#pragma unroll
        for (int q = 0; q < NC; ++q) win[q] = 0.0;
        for (int r = N - 1; r >= 0; --r) {
            double v = x[r];
#pragma unroll
            for (int q = 1; q <= NC; ++q)
                if (r + q < N) v -= fac[static_cast<size_t>((r + q) * W + q) * cs + i] * win[q - 1];
            const double xr = v * fac[static_cast<size_t>(r * W) * cs + i];
            x[r] = xr;
#pragma unroll
            for (int q = NC - 1; q > 0; --q) win[q] = win[q - 1];
            win[0] = xr;
            if constexpr (MX) reinterpret_cast<float*>(L0.u)[r] = narrow(xr);  // FP32 copy for the first FMG interpolation
        }
        double F0;
        if (A.qoi == MLQMC_QOI_MEAN) {
            double acc = 0.0;
            for (int r = 0; r < N; ++r) acc += x[r];
            F0 = acc / static_cast<double>(N);
        } else {
            constexpr int m = NC / 2;
            F0 = 0.25 * (x[(m - 1) * NC + (m - 1)] + x[(m - 1) * NC + m] + x[m * NC + (m - 1)] + x[m * NC + m]);
        }
        A.F[static_cast<size_t>(i) * A.n_levels] = F0;
    }
}

// Level 0 for n0 = NC for calls of few samples: the same factorisation,
// substitutions and F_0 as kb_level0_fixed, every operation in its order, but
// each step of the factorisation split over the NC + 2 warps of a CTA that
// holds 32 samples (lane = sample). On GB300 an FP64 warp instruction holds
// its SM sub-partition for about 70 cycles whatever its active lanes, so one
// thread's ~4,700 FP64 operations take 0.15 ms or more however few samples a
// call has. Split this way a step's FP64 work runs on several sub-partitions
// at once; what remains per step is the dependent chain of the reciprocal
// square root and the shared FP64 pipes (about 0.18 ms per call). Step j:
// warp 0 forms d_j and 1/L(j,j) (the face sum of d_j formed one step ahead by
// warp NC, whose band row is the shortest), warp l (1..NC) the dot product of
// row j+l, warp NC+1 the forward value; after a barrier warp l scales its entry of
// column j, warp NC+1 finishes y_j and warp 0 writes the finished row j to
// the global factor; a second barrier ends the step. Warp NC+1 then runs the
// backward substitution (the factor rows from global memory, written by warp
// 0 before the barriers) and forms F_0. The ring of NC+1 rows and the
// forward values of the group's samples sit in shared memory. Lanes past B
// compute on sample B-1 and store nothing.
template <typename T, bool MX, int NC>
__global__ void __launch_bounds__(32 * (NC + 2)) kb_level0_split(FmgArgs A, int B)
{
    constexpr int N = NC * NC, W = NC + 1;
    __shared__ double ring[W * W * 32];  // [(slot * W + e) * 32 + lane]
    __shared__ double ys[N * 32];        // forward values, then the solution
    __shared__ double dg[2 * 32];        // the diagonal sum of the next step, formed one step ahead
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t cs = A.chol.stride;
    double* fac = reinterpret_cast<double*>(A.chol.base);
    float* f32 = reinterpret_cast<float*>(A.chol32);
    const double h2 = 1.0 / (static_cast<double>(NC) * NC);
    auto Rs = [&](int slot, int e) -> double& { return ring[(slot * W + e) * 32 + lane]; };
    for (int base = blockIdx.x * 32; base < B; base += gridDim.x * 32) {
        const int i = base + lane;
        const bool live = i < B;
        const int si = live ? i : B - 1;
        const Lv<T> L0 = view<T>(A, 0, si);
        double win[NC];  // forward substitution: win[q - 1] = y_(j - q)
#pragma unroll
        for (int q = 0; q < NC; ++q) win[q] = 0.0;
        auto step = [&](int j, auto full) {
            constexpr bool FULL = decltype(full)::value;
            const int s0 = j % W;
            double a = 0.0, v = 0.0;
            int sr = 0;
            const int l = warp;  // row j + l for warps 1..NC
            // the face sum of row jj's diagonal, in kb_level0_fixed's order
            auto diag_sum = [&](int jj) {
                const int j1 = jj % NC, j2 = jj / NC;
                return widen(L0.kx[j2 * kx_pitch(NC) + j1]) + widen(L0.kx[j2 * kx_pitch(NC) + j1 + 1]) +
                       widen(L0.ky[j2 * NC + j1]) + widen(L0.ky[(j2 + 1) * NC + j1]);
            };
            if (warp == 0) {
                double d = j == 0 ? diag_sum(0) : dg[(j & 1) * 32 + lane];  // step j > 0: formed by warp NC
#pragma unroll
                for (int q = 1; q <= NC; ++q) {
                    if (!FULL && q > j) break;
                    const double lq = Rs(s0, q);
                    d -= lq * lq;
                }
                Rs(s0, 0) = rsqrt64(d);
            } else if (warp <= NC) {
                if (warp == NC && j + 1 < N) dg[((j + 1) & 1) * 32 + lane] = diag_sum(j + 1);  // the lightest row's warp
                const int r = j + l;
                if (r < N) {
                    sr = s0 + l >= W ? s0 + l - W : s0 + l;
                    a = widen(band_a(L0.kx, L0.ky, NC, r, l));
                    if constexpr (FULL) {
                        for (int u = 0; u < NC - l; ++u) a -= Rs(sr, NC - u) * Rs(s0, NC - l - u);
                    } else {
                        for (int tt = (r - NC > 0 ? r - NC : 0); tt < j; ++tt) a -= Rs(sr, r - tt) * Rs(s0, j - tt);
                    }
                }
            } else {
                v = h2;  // forward substitution, f = 1
#pragma unroll
                for (int q = 1; q <= NC; ++q) {
                    if (!FULL && q > j) break;
                    v -= Rs(s0, q) * win[q - 1];
                }
            }
            __syncthreads();
            const double rl = Rs(s0, 0);
            if (warp == 0) {
                if (live) {
#pragma unroll
                    for (int e = 0; e <= NC; ++e) {
                        if (!FULL && e > j) break;
                        fac[static_cast<size_t>(j * W + e) * cs + i] = Rs(s0, e);
                        if constexpr (MX) f32[static_cast<size_t>(j * W + e) * cs + i] = narrow(Rs(s0, e));
                    }
                }
            } else if (warp <= NC) {
                if (j + l < N) Rs(sr, l) = a * rl;
            } else {
                const double yj = v * rl;
                ys[j * 32 + lane] = yj;
#pragma unroll
                for (int q = NC - 1; q > 0; --q) win[q] = win[q - 1];
                win[0] = yj;
            }
            __syncthreads();
        };
        for (int j = 0; j < NC; ++j) step(j, std::false_type());
        for (int j = NC; j < N; ++j) step(j, std::true_type());
        if (warp == NC + 1) {
            // backward: x_r = (y_r - sum_q L(r+q, r) x_(r+q)) / L(r, r), win[q - 1] = x_(r+q)
            double* x = (MX || A.refine) ? L0.u64 : reinterpret_cast<double*>(L0.u);
#pragma unroll
            for (int q = 0; q < NC; ++q) win[q] = 0.0;
            for (int r = N - 1; r >= 0; --r) {
                double v = ys[r * 32 + lane];
#pragma unroll
                for (int q = 1; q <= NC; ++q)
                    if (r + q < N) v -= fac[static_cast<size_t>((r + q) * W + q) * cs + si] * win[q - 1];
                const double xr = v * fac[static_cast<size_t>(r * W) * cs + si];
                ys[r * 32 + lane] = xr;
                if (live) {
                    x[r] = xr;
                    if constexpr (MX) reinterpret_cast<float*>(L0.u)[r] = narrow(xr);  // FP32 copy for the first FMG interpolation
                }
#pragma unroll
                for (int q = NC - 1; q > 0; --q) win[q] = win[q - 1];
                win[0] = xr;
            }
            double F0;
            if (A.qoi == MLQMC_QOI_MEAN) {
                double acc = 0.0;
                for (int r = 0; r < N; ++r) acc += ys[r * 32 + lane];
                F0 = acc / static_cast<double>(N);
            } else {
                constexpr int m = NC / 2;
                F0 = 0.25 * (ys[((m - 1) * NC + (m - 1)) * 32 + lane] + ys[((m - 1) * NC + m) * 32 + lane] +
                             ys[(m * NC + (m - 1)) * 32 + lane] + ys[(m * NC + m) * 32 + lane]);
            }
            if (live) A.F[static_cast<size_t>(i) * A.n_levels] = F0;
        }
        __syncthreads();
    }
}

template <int NC>
constexpr size_t level0_smem()
{
    return sizeof(double) * static_cast<size_t>((NC + 1) * (NC + 1)) * 64;
}

// Coarse solve for n0 = NC fixed at compile time: a CTA of 64 threads takes 64
// consecutive samples, stages their right-hand sides transposed in shared
// memory (coalesced loads; row pitch 65 avoids bank conflicts), solves one
// sample per thread with the factor rows prefetched PF rows ahead, and writes
// the solutions back coalesced.
template <typename T, int NC>
__global__ void __launch_bounds__(64) kb_coarse_fixed(FmgArgs A, int B)
{
    // rows prefetched ahead: each group of PF rows costs one memory latency (FP64: 190 registers, no spills)
    constexpr int N = NC * NC, W = NC + 1, P = 65, PF = 8;
    __shared__ T xs[N * P];
    const T h2 = T(1) / (T(NC) * T(NC));
    const T* fac = reinterpret_cast<const T*>(sizeof(T) == 4 ? A.chol32 : A.chol.base);
    const size_t cs = A.chol.stride;
    for (int base = blockIdx.x * 64; base < B; base += gridDim.x * 64) {
        const int cnt = B - base < 64 ? B - base : 64;
        for (int q = threadIdx.x; q < cnt * N; q += 64) {
            const int j = q / N, r = q - j * N;
            xs[r * P + j] = h2 * at<T>(A.lv[0].bc, base + j)[r];
        }
        __syncthreads();
        const int j = threadIdx.x;
        const int i = base + j;
        if (j < cnt && !(A.active && !A.active[i])) {
            T* x = xs + j;
            T ring[PF][W];
#pragma unroll
            for (int a = 0; a < PF; ++a)
#pragma unroll
                for (int q = 0; q < W; ++q) ring[a][q] = fac[static_cast<size_t>(a * W + q) * cs + i];
            for (int r0 = 0; r0 < N; r0 += PF) {
#pragma unroll
                for (int a = 0; a < PF; ++a) {
                    const int r = r0 + a;
                    T v = x[r * P];
#pragma unroll
                    for (int q = NC; q >= 1; --q)
                        if (q <= r) v -= ring[a][q] * x[(r - q) * P];
                    x[r * P] = v * ring[a][0];
                    if (r + PF < N) {
#pragma unroll
                        for (int q = 0; q < W; ++q) ring[a][q] = fac[static_cast<size_t>((r + PF) * W + q) * cs + i];
                    }
                }
            }
            // backward: x_r -= sum_q L(r+q, r) x_{r+q}, entry (r+q, q)
            for (int r0 = N - 1; r0 >= 0; r0 -= PF) {
#pragma unroll
                for (int a = 0; a < PF; ++a) {
                    const int r = r0 - a;
                    if (r < 0) break;
                    T v = x[r * P];
#pragma unroll
                    for (int q = NC; q >= 1; --q)
                        if (r + q < N) v -= fac[static_cast<size_t>((r + q) * W + q) * cs + i] * x[(r + q) * P];
                    x[r * P] = v * fac[static_cast<size_t>(r * W) * cs + i];
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * N; q += 64) {
            const int jj = q / N, r = q - jj * N;
            if (!(A.active && !A.active[base + jj])) at<T>(A.lv[0].u, base + jj)[r] = xs[r * P + jj];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Level-synchronous kernels over samples 0..B-1 of level t.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool inactive(const FmgArgs& A, int i)
{
    return A.active && !A.active[i];
}

// G[i][a][i2] = sum_{m: a_m = a} sqrt(theta_m) y_m psi_{b_m}(x2)
template <typename T>
__global__ void kb_synth_G(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const T* psi = static_cast<const T*>(A.psi) + A.psi_off[t];
    const uint32_t per = static_cast<uint32_t>(A.Ka) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_kan.div(idx));
        const int rem = static_cast<int>(idx - i * per);
        const int a = static_cast<int>(A.lv[t].by_n.div(rem));
        const int i2 = rem - a * n;
        T acc = T(0);
        const int g1 = A.grp_start[a + 1];
        if constexpr (sizeof(T) == 4) {
            // FP32 coefficients sqrt(theta_m) y_m from k_coef32 (the same rounded products)
            const float* cf = A.c32 + static_cast<size_t>(i) * A.s;
            for (int g = A.grp_start[a]; g < g1; ++g) acc += cf[A.grp_m[g]] * psi[A.grp_b[g] * n + i2];
        } else {
            const double* y = A.Y + static_cast<size_t>(A.samples[i].canon) * A.s;
            for (int g = A.grp_start[a]; g < g1; ++g) acc += (A.grp_sqrt[g] * y[A.grp_m[g]]) * psi[A.grp_b[g] * n + i2];
        }
        at<T>(A.lv[t].G, i)[rem] = acc;
    }
}

// Mixed forms: c32[i][m] = sqrt(theta_m) y_m of sample i (rank order) rounded
// to FP32, once per launch of the FP32 separable synthesis, so that its inner
// loop issues no FP64 operation.
__global__ void k_coef32(FmgArgs A, int B, const double* __restrict__ sq, float* __restrict__ out)
{
    const int64_t total = static_cast<int64_t>(B) * A.s;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(idx / A.s);
        const int m = static_cast<int>(idx - static_cast<int64_t>(i) * A.s);
        out[idx] = narrow(sq[m] * A.Y[static_cast<size_t>(A.samples[i].canon) * A.s + m]);
    }
}

// k = exp(sum_a psi_a(x1) G_a(x2))
template <typename T>
__global__ void kb_synth_z(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const T* psi = static_cast<const T*>(A.psi) + A.psi_off[t];
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        const int p = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_n.div(p));
        const int i1 = p - i2 * n;
        const T* G = at<T>(A.lv[t].G, i);
        T z = T(0);
        for (int a = 0; a < A.Ka; ++a) z += psi[a * n + i1] * G[a * n + i2];
        at<T>(A.lv[t].k, i)[p] = expT(z);
    }
}

// Matern modes: z(x_p) = sum_j Psi_t(x_p, j) sqrt(theta_j) y_j (eq.
// truncatedKL with the level's interpolated Nystrom modes), k = exp(z), the
// sum in FP64. A thread takes one cell and kG samples, so each row of Psi_t
// is read once per kG samples; the kG samples' coefficients sqrt(theta_j) y_j
// are staged in shared memory, kJ modes at a time.
constexpr int kDenseG = 8, kDenseJ = 512;
template <typename T>
__global__ void __launch_bounds__(256) kb_synth_dense(FmgArgs A, int t, int B, const double* __restrict__ psi, int s,
                                                      const double* __restrict__ sq)
{
    __shared__ double cs[kDenseG][kDenseJ];
    const int n = A.lv[t].n;
    const int ncell = n * n;
    const int i0 = blockIdx.y * kDenseG;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[kDenseG];
#pragma unroll
    for (int g = 0; g < kDenseG; ++g) acc[g] = 0.0;
    for (int j0 = 0; j0 < s; j0 += kDenseJ) {
        const int jn = min(kDenseJ, s - j0);
        for (int e = threadIdx.x; e < kDenseG * kDenseJ; e += blockDim.x) {
            const int g = e / kDenseJ, jj = e - g * kDenseJ;
            const int i = i0 + g;
            cs[g][jj] = (i < B && jj < jn) ? sq[j0 + jj] * A.Y[static_cast<size_t>(A.samples[i].canon) * A.s + j0 + jj]
                                           : 0.0;
        }
        __syncthreads();
        if (p < ncell) {
            const double* row = psi + static_cast<size_t>(p) * s + j0;
            for (int jj = 0; jj < jn; ++jj) {
                const double v = row[jj];
#pragma unroll
                for (int g = 0; g < kDenseG; ++g) acc[g] = fma(v, cs[g][jj], acc[g]);
            }
        }
        __syncthreads();
    }
    if (p < ncell) {
#pragma unroll
        for (int g = 0; g < kDenseG; ++g)
            if (i0 + g < B) at<T>(A.lv[t].k, i0 + g)[p] = expT(static_cast<T>(acc[g]));
    }
}

template <typename T>
__global__ void kb_faces(FmgArgs A, int t, int B)
{
    // one cell per thread: its west x face and north y face, plus the east
    // boundary face in the last column and the south one in the last row
    const int n = A.lv[t].n;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        const int p = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_n.div(p));
        const int i1 = p - i2 * n;
        const T* k = at<T>(A.lv[t].k, i);
        T* kx = at<T>(A.lv[t].kx, i) + i2 * kx_pitch(n);
        T* ky = at<T>(A.lv[t].ky, i);
        kx[i1] = face_x(k, n, i2, i1);
        if (i1 == n - 1) kx[n] = face_x(k, n, i2, n);
        ky[i2 * n + i1] = face_y(k, n, i2, i1);
        if (i2 == n - 1) ky[n * n + i1] = face_y(k, n, n, i1);
    }
}

// FP32 faces, four cells of a row per thread (16-byte loads and stores; n a
// multiple of 4): the west x faces and north y faces of cells i1..i1+3 of row
// i2, the east boundary face after the last column and the south boundary
// faces below the last row. The arithmetic of face_x / face_y, operand for
// operand.
__global__ void kb_faces4(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const int q = n >> 2;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(q);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nnq.div(idx));
        const int p4 = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_nq.div(p4));
        const int i1 = (p4 - i2 * q) * 4;
        const float* k = at<float>(A.lv[t].k, i);
        float* kx = at<float>(A.lv[t].kx, i) + i2 * kx_pitch(n);
        float* ky = at<float>(A.lv[t].ky, i);
        const float4 c = *reinterpret_cast<const float4*>(k + i2 * n + i1);
        const float4 fx = make_float4(i1 > 0 ? hmean(k[i2 * n + i1 - 1], c.x) : 2.0f * c.x, hmean(c.x, c.y),
                                      hmean(c.y, c.z), hmean(c.z, c.w));
        *reinterpret_cast<float4*>(kx + i1) = fx;
        if (i1 + 4 == n) kx[n] = 2.0f * c.w;
        float4 fy;
        if (i2 > 0) {
            const float4 a = *reinterpret_cast<const float4*>(k + (i2 - 1) * n + i1);
            fy = make_float4(hmean(a.x, c.x), hmean(a.y, c.y), hmean(a.z, c.z), hmean(a.w, c.w));
        } else {
            fy = make_float4(2.0f * c.x, 2.0f * c.y, 2.0f * c.z, 2.0f * c.w);
        }
        *reinterpret_cast<float4*>(ky + i2 * n + i1) = fy;
        if (i2 == n - 1)
            *reinterpret_cast<float4*>(ky + n * n + i1) = make_float4(2.0f * c.x, 2.0f * c.y, 2.0f * c.z, 2.0f * c.w);
    }
}

template <typename T>
__global__ void kb_idiag(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        const int p = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_n.div(p));
        at<T>(A.lv[t].idiag, i)[p] = inv_diag(at<T>(A.lv[t].kx, i), at<T>(A.lv[t].ky, i), n, p - i2 * n, i2);
    }
}

// One colour of a red-black sweep; ones: right-hand side 1, else bc of level t.
template <typename T>
__global__ void kb_gs(FmgArgs A, int t, int B, int colour, int ones)
{
    const int n = A.lv[t].n;
    const int half = n >> 1;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(half);
    const T h2 = T(1) / (T(n) * T(n));
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nnc.div(idx));
        if (inactive(A, i)) continue;
        const int q = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_nc.div(q));
        const Lv<T> L = view<T>(A, t, i);
        gs_cell(L, ones ? nullptr : L.bc, h2, 2 * (q - i2 * half) + ((i2 + colour) & 1), i2);
    }
}

// NS full red-black sweeps of one TILE x TILE tile per CTA iteration (temporal
// blocking): u, 1/D and b are staged in shared memory with a halo of H cells
// on each side (16-byte loads from 16-byte aligned rows, zeros outside the
// domain, which is the Dirichlet ghost value), the x and y faces of the same
// region too; the NS sweeps consume 2*NS of that halo. FP32 (mixed forms) and
// FP64 (FP64 form, one sweep per launch: FP64 arithmetic is the scarce
// resource on GB300, so the halo is kept at the 2 cells one sweep consumes).
// u is read from u and written to u2 (ping-pong, so no tile reads a
// neighbour's half-updated cells). Phase p updates its colour on the tile
// grown by 2*NS-1-p with the operations of gs_cell in its order (an outside
// neighbour is a staged zero, whose product adds exactly nothing); the result
// equals NS passes of kb_gs over both colours, bit for bit.
// first: colour of the first half sweep (0 red for pre-smoothing, 1 black).
// PROLONG: the staged u first receives the coarse-grid correction P e from
// level t-1 (post-smoothing of the V-cycle), as kb_prolong would add it.
template <typename T, int NS>
struct TileHalo {
    static constexpr int H = (sizeof(T) == 8 && NS == 1) ? 2 : 4;  // x0 - H stays 16-byte aligned
};

template <typename T, int TILE, int NS, bool PROLONG>
__global__ void __launch_bounds__(256) kb_rbgs_tile(FmgArgs A, int t, int B, int ones, int first)
{
    static_assert(NS == 1 || NS == 2, "one or two sweeps per launch");
    using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int VW = 16 / static_cast<int>(sizeof(T));  // elements per 16-byte vector
    constexpr int H = TileHalo<T, NS>::H;                  // staged halo
    constexpr int HN = 2 * NS;                             // halo the NS sweeps consume
    constexpr int SU = TILE + 2 * H;                       // staged side
    constexpr int V = SU / VW;                             // vectors per staged row
    static_assert(SU % VW == 0 && H % VW == 0 && H >= HN, "staged rows are whole 16-byte vectors");
    extern __shared__ float4 smraw4[];
    T* su = reinterpret_cast<T*>(smraw4);  // SU x SU
    T* sid = su + SU * SU;                 // SU x SU
    T* sb = sid + SU * SU;                 // SU x SU
    T* sky = sb + SU * SU;                 // (SU + 1) face rows x SU
    T* skx = sky + (SU + 1) * SU;          // SU rows x (SU + 1) faces
    const int n = A.lv[t].n;
    const int tx_n = n / TILE;
    const uint32_t per = static_cast<uint32_t>(tx_n) * static_cast<uint32_t>(tx_n);
    const T h2 = T(1) / (static_cast<T>(n) * static_cast<T>(n));
    V16 z4, o4;
    {
        T* zp = reinterpret_cast<T*>(&z4);
        T* op = reinterpret_cast<T*>(&o4);
#pragma unroll
        for (int j = 0; j < VW; ++j) zp[j] = T(0), op[j] = T(1);
    }
    for (int64_t tile = blockIdx.x; tile < B * per; tile += gridDim.x) {
        const int i = static_cast<int>(tile / per);
        if (inactive(A, i)) continue;
        const int tr = static_cast<int>(tile - i * per);
        const int y0 = (tr / tx_n) * TILE, x0 = (tr % tx_n) * TILE;
        const Lv<T> L = view<T>(A, t, i);
        T* uo = at<T>(A.lv[t].u2, i);
        // cell arrays: rows y0-H.., columns x0-H.. in 16-byte vectors (x0-H is a multiple of VW)
#pragma unroll 4
        for (int q = threadIdx.x; q < SU * V; q += blockDim.x) {
            const int r = q / V, v = q - (q / V) * V;
            const int gy = y0 - H + r, gx = x0 - H + VW * v;
            const bool in = gy >= 0 && gy < n && gx >= 0 && gx < n;
            const size_t o = static_cast<size_t>(gy) * n + gx;
            reinterpret_cast<V16*>(su)[q] = in ? *reinterpret_cast<const V16*>(L.u + o) : z4;
            reinterpret_cast<V16*>(sid)[q] = in ? *reinterpret_cast<const V16*>(L.idiag + o) : z4;
            reinterpret_cast<V16*>(sb)[q] = in ? (ones ? o4 : *reinterpret_cast<const V16*>(L.bc + o)) : z4;
        }
        if constexpr (PROLONG) {
            // coarse-grid correction first: u += P e on every staged cell of the domain
            __syncthreads();
            const T* e = at<T>(A.lv[t - 1].u, i);
            const int nc = n >> 1;
            for (int q = threadIdx.x; q < SU * SU; q += blockDim.x) {
                const int gy = y0 - H + q / SU, gx = x0 - H + q % SU;
                if (gy >= 0 && gy < n && gx >= 0 && gx < n) su[q] += prolong_cell<T, T>(e, nc, gx, gy);
            }
        }
        // y faces: face rows y0-H .. y0-H+SU, columns as above
#pragma unroll 4
        for (int q = threadIdx.x; q < (SU + 1) * V; q += blockDim.x) {
            const int r = q / V, v = q - (q / V) * V;
            const int gy = y0 - H + r, gx = x0 - H + VW * v;
            const bool in = gy >= 0 && gy <= n && gx >= 0 && gx < n;
            reinterpret_cast<V16*>(sky)[q] =
                in ? *reinterpret_cast<const V16*>(L.ky + static_cast<size_t>(gy) * n + gx) : z4;
        }
        // x faces: rows y0-H.., faces x0-H .. x0-H+SU (row pitch kx_pitch(n): scalar loads)
#pragma unroll 4
        for (int q = threadIdx.x; q < SU * (SU + 1); q += blockDim.x) {
            const int r = q / (SU + 1), f = q - (q / (SU + 1)) * (SU + 1);
            const int gy = y0 - H + r, gx = x0 - H + f;
            skx[q] = (gy >= 0 && gy < n && gx >= 0 && gx <= n) ? L.kx[static_cast<size_t>(gy) * kx_pitch(n) + gx]
                                                                : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int ph = 0; ph < HN; ++ph) {
            const int colour = (first + ph) & 1;
            const int g = HN - 1 - ph;  // growth of the updated region beyond the tile
            const int side = TILE + 2 * g;
            const int half = side / 2;
            for (int q = threadIdx.x; q < side * half; q += blockDim.x) {
                const int ry = q / half;
                const int gy = y0 - g + ry;
                const int rx = 2 * (q - ry * half) + ((gy + x0 - g + colour) & 1);
                const int gx = x0 - g + rx;
                if (gy < 0 || gy >= n || gx < 0 || gx >= n) continue;
                const int sy = gy - y0 + H, sx = gx - x0 + H;
                const int c0 = sy * SU + sx;
                const T* kr = skx + sy * (SU + 1);
                T acc = h2 * sb[c0];
                acc += kr[sx] * su[c0 - 1];
                acc += kr[sx + 1] * su[c0 + 1];
                acc += sky[sy * SU + sx] * su[c0 - SU];
                acc += sky[(sy + 1) * SU + sx] * su[c0 + SU];
                su[c0] = acc * sid[c0];
            }
            __syncthreads();
        }
        constexpr int TV = TILE / VW;
        for (int q = threadIdx.x; q < TILE * TV; q += blockDim.x) {
            const int ry = q / TV, v = q - (q / TV) * TV;
            const T* src = su + (ry + H) * SU + H + VW * v;
            V16 w;
            T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
            for (int j = 0; j < VW; ++j) wp[j] = src[j];
            *reinterpret_cast<V16*>(uo + static_cast<size_t>(y0 + ry) * n + x0 + VW * v) = w;
        }
        __syncthreads();
    }
}

// bc of level t-1 = mean over children of (b - A u) on level t.
template <typename T>
__global__ void kb_resid_restrict(FmgArgs A, int t, int B, int ones)
{
    const int nc = A.lv[t].n >> 1;
    const uint32_t per = static_cast<uint32_t>(nc) * static_cast<uint32_t>(nc);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_ncnc.div(idx));
        if (inactive(A, i)) continue;
        const int q = static_cast<int>(idx - i * per);
        const int I2 = static_cast<int>(A.lv[t].by_nc.div(q));
        const Lv<T> F = view<T>(A, t, i);
        at<T>(A.lv[t - 1].bc, i)[q] = resid_restrict_cell(F, ones ? nullptr : F.bc, q - I2 * nc, I2);
    }
}

// The 2 x 2 fine cells of coarse parent (I1, I2) receive P e (the arithmetic
// of prolong_cell): the parent's 3 x 3 coarse neighbourhood, a neighbour
// outside the coarse grid replaced by minus the parent's row or column (odd
// reflection; the corner by the product of the two signs). dst(fx, fy) of
// the block at rows 2 I2 + fy, columns 2 I1 + fx.
template <typename S, typename D, typename Store>
__device__ __forceinline__ void prolong_block(const S* e, int nc, int I1, int I2, Store store)
{
    const bool lo1 = I1 == 0, hi1 = I1 == nc - 1, lo2 = I2 == 0, hi2 = I2 == nc - 1;
    D E[3][3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const bool ry = (dy < 0 && lo2) || (dy > 0 && hi2);
            const bool rx = (dx < 0 && lo1) || (dx > 0 && hi1);
            const D v = D(e[(I2 + (ry ? 0 : dy)) * nc + I1 + (rx ? 0 : dx)]);
            E[dy + 1][dx + 1] = (ry != rx) ? -v : v;
        }
    }
    D out[2][2];
#pragma unroll
    for (int fy = 0; fy < 2; ++fy)
#pragma unroll
        for (int fx = 0; fx < 2; ++fx)
            out[fy][fx] = fma(D(0.5625), E[1][1], fma(D(0.1875), E[1][2 * fx] + E[2 * fy][1], D(0.0625) * E[2 * fy][2 * fx]));
    store(out);
}

// u of level t (+)= P u of level t-1 (FP64 solution arrays when U64), one
// coarse parent (2 x 2 fine cells) per thread.
template <typename T, bool ADD, bool U64>
__global__ void kb_prolong(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const int nc = n >> 1;
    const uint32_t per = static_cast<uint32_t>(nc) * static_cast<uint32_t>(nc);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_ncnc.div(idx));
        if (inactive(A, i)) continue;
        const int q = static_cast<int>(idx - i * per);
        const int I2 = static_cast<int>(A.lv[t].by_nc.div(q));
        const int I1 = q - I2 * nc;
        const size_t o = static_cast<size_t>(2 * I2) * n + 2 * I1;
        if constexpr (U64) {
            // FMG interpolation of the refinement path into u64: mixed forms
            // interpolate the FP32 copy of the coarse solution in FP32 (the
            // first FP64 residual then sees it exactly), FP64 form in FP64
            double* u = at<double>(A.lv[t].u64, i) + o;
            auto store = [&](const auto& v) {
#pragma unroll
                for (int fy = 0; fy < 2; ++fy) {
                    double2* d = reinterpret_cast<double2*>(u + fy * n);
                    const double2 w = make_double2(widen(v[fy][0]), widen(v[fy][1]));
                    if (ADD) *d = make_double2(d->x + w.x, d->y + w.y);
                    else *d = w;
                }
            };
            if constexpr (sizeof(T) == 4) prolong_block<float, float>(at<float>(A.lv[t - 1].u, i), nc, I1, I2, store);
            else prolong_block<double, double>(at<double>(A.lv[t - 1].u64, i), nc, I1, I2, store);
        } else {
            T* u = at<T>(A.lv[t].u, i) + o;
            prolong_block<T, T>(at<T>(A.lv[t - 1].u, i), nc, I1, I2, [&](const T (&v)[2][2]) {
#pragma unroll
                for (int fy = 0; fy < 2; ++fy) {
                    T* d = u + fy * n;
                    d[0] = ADD ? d[0] + v[fy][0] : v[fy][0];
                    d[1] = ADD ? d[1] + v[fy][1] : v[fy][1];
                }
            });
        }
    }
}

// Refinement path: bc = 1 - A u64 (FP64 residual, working-precision faces widened).
template <typename T>
__global__ void kb_resid64(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    const double ih2 = static_cast<double>(n) * n;
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        if (inactive(A, i)) continue;
        const int p = static_cast<int>(idx - i * per);
        const int i2 = static_cast<int>(A.lv[t].by_n.div(p));
        const Lv<T> L = view<T>(A, t, i);
        L.bc[p] = to_work<T>(resid64_cell(L, ih2, p - i2 * n, i2));
    }
}

// Mixed forms, the refinement step that opens level t: the FMG interpolation
// u64 = P u_(t-1) (of the FP32 copy of the coarse solution, in FP32: the
// arithmetic of kb_prolong) and r = 1 - A u64 in one pass, each cell
// interpolating its own value and its four neighbours'. Every input of this
// residual is an FP32 number (u64 holds the widened FP32 interpolant), so it
// is formed with FP32 error-free transformations (resid_f32x2) to within a
// few units of 2^-48 of the terms, as accurate as the FP64 evaluation of
// kb_resid64 before r is rounded to FP32, and without the FP64 pipe.
__global__ void __launch_bounds__(256, 4) kb_prolong_resid64(FmgArgs A, int t, int B)
{
    // one thread per coarse cell (I1, I2), i.e. per 2 x 2 quad of fine cells:
    // the quad and its ring of 8 fine neighbours all interpolate from the
    // 3 x 3 coarse block around (I1, I2), odd-reflected across the boundary as
    // in prolong_cell (a fine cell's out-of-range coarse neighbour is minus
    // the value in its parent's own row or column)
    const int n = A.lv[t].n, nc = n >> 1;
    const uint32_t per = static_cast<uint32_t>(nc) * static_cast<uint32_t>(nc);
    const float ih2 = static_cast<float>(n) * static_cast<float>(n);  // exact: n = coarse_cells 2^t
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_ncnc.div(idx));
        if (inactive(A, i)) continue;
        const int q = static_cast<int>(idx - i * per);
        const int I2 = static_cast<int>(A.lv[t].by_nc.div(q)), I1 = q - I2 * nc;
        const float* e = at<float>(A.lv[t - 1].u, i);
        const Lv<float> L = view<float>(A, t, i);
        // the quad's faces, loaded before any store of this iteration
        float2 kx01[2], kyn[2], kys[2];
        float kx2[2];
#pragma unroll
        for (int qy = 0; qy < 2; ++qy) {
            const int i1 = 2 * I1, i2 = 2 * I2 + qy;
            const float* kxr = L.kx + i2 * kx_pitch(n) + i1;
            kx01[qy] = *reinterpret_cast<const float2*>(kxr);
            kx2[qy] = kxr[2];
            kyn[qy] = *reinterpret_cast<const float2*>(L.ky + i2 * n + i1);
            kys[qy] = *reinterpret_cast<const float2*>(L.ky + (i2 + 1) * n + i1);
        }
        float E[3][3];  // E[dy + 1][dx + 1]
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = I1 + dx, y = I2 + dy;
                const bool ox = x < 0 || x >= nc, oy = y < 0 || y >= nc;
                const float v = e[(oy ? I2 : y) * nc + (ox ? I1 : x)];
                E[dy + 1][dx + 1] = (ox != oy) ? -v : v;
            }
        // fine cells 2I + f, f = -1..2 per axis (the four ring corners unused):
        // parent offset (f - 1) / 2 rounded down, coarse neighbour towards the
        // cell's side (+1 for odd f, -1 for even f); cells outside the grid are 0
        float U[4][4];
#pragma unroll
        for (int fy = -1; fy <= 2; ++fy)
#pragma unroll
            for (int fx = -1; fx <= 2; ++fx) {
                const bool ring_x = fx < 0 || fx > 1, ring_y = fy < 0 || fy > 1;
                if (ring_x && ring_y) {
                    U[fy + 1][fx + 1] = 0.0f;
                    continue;
                }
                const int i1 = 2 * I1 + fx, i2 = 2 * I2 + fy;
                if (i1 < 0 || i1 >= n || i2 < 0 || i2 >= n) {
                    U[fy + 1][fx + 1] = 0.0f;
                    continue;
                }
                const int px = fx < 0 ? -1 : (fx > 1 ? 1 : 0), py = fy < 0 ? -1 : (fy > 1 ? 1 : 0);
                const int sx = (fx & 1) ? 1 : -1, sy = (fy & 1) ? 1 : -1;
                const float a = E[py + 1][px + 1];
                const float bx = E[py + 1][px + sx + 1];
                const float cy = E[py + sy + 1][px + 1];
                const float d = E[py + sy + 1][px + sx + 1];
                U[fy + 1][fx + 1] = fmaf(0.5625f, a, fmaf(0.1875f, bx + cy, 0.0625f * d));
            }
        // residual of each quad cell: every input an FP32 number (pairs, as resid_f32x2 states);
        // a quad row's two cells are adjacent: their faces are loaded and their
        // u64 and b written as pairs (16- and 8-byte accesses; i1 even, pitches even)
#pragma unroll
        for (int qy = 0; qy < 2; ++qy) {
            const int i1 = 2 * I1, i2 = 2 * I2 + qy;
            const int p = i2 * n + i1;
            float r[2];
#pragma unroll
            for (int qx = 0; qx < 2; ++qx) {
                const float up = U[qy + 1][qx + 1];
                const float uv[4] = {U[qy + 1][qx], U[qy + 1][qx + 2], U[qy][qx + 1], U[qy + 2][qx + 1]};
                const float kv[4] = {qx ? kx01[qy].y : kx01[qy].x, qx ? kx2[qy] : kx01[qy].y,
                                     qx ? kyn[qy].y : kyn[qy].x, qx ? kys[qy].y : kys[qy].x};
                r[qx] = resid_f32x2(kv, up, uv, ih2);
            }
            *reinterpret_cast<double2*>(L.u64 + p) = make_double2(widen(U[qy + 1][1]), widen(U[qy + 1][2]));
            *reinterpret_cast<float2*>(L.bc + p) = make_float2(r[0], r[1]);
        }
    }
}

// Refinement path: u64 += e.
template <typename T>
__global__ void kb_update64(FmgArgs A, int t, int B)
{
    const int n = A.lv[t].n;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        if (inactive(A, i)) continue;
        const int p = static_cast<int>(idx - i * per);
        at<double>(A.lv[t].u64, i)[p] += widen(at<T>(A.lv[t].u, i)[p]);
    }
}

// Refinement residual r = 1 - A u64 of level t (left in bc for the next correction)
// with the cells of each sample in P contiguous chunks, one CTA per (sample,
// chunk), so that a few large samples still fill the GPU: part[i * P + q] =
// the chunk's sum of r^2 (fixed order inside the CTA).
template <typename T>
__global__ void __launch_bounds__(256) kb_resnorm_part(FmgArgs A, int t, int B, int P, double* part)
{
    __shared__ double red[48];
    const int n = A.lv[t].n;
    const int nn = n * n;
    const int csz = (nn + P - 1) / P;
    const double ih2 = static_cast<double>(n) * n;
    for (int w = blockIdx.x; w < B * P; w += gridDim.x) {  // uniform per CTA: every thread reaches block_sum
        const int i = w / P, q = w - i * P;
        const Lv<T> L = view<T>(A, t, i);
        const int p1 = min(nn, (q + 1) * csz);
        double acc = 0.0;
        for (int p = q * csz + static_cast<int>(threadIdx.x); p < p1; p += blockDim.x) {
            const int i2 = static_cast<int>(A.lv[t].by_n.div(p));
            const double r = resid64_cell(L, ih2, p - i2 * n, i2);
            L.bc[p] = to_work<T>(r);
            acc += r * r;
        }
        const double sum = block_sum(acc, red);
        if (threadIdx.x == 0) part[w] = sum;
    }
}

// norms[i] = sqrt of the sum of sample i's P partial sums (in chunk order),
// active[i] = (norm_i > thresh); *count = number of active samples.
__global__ void kb_norm_flags(const double* part, int P, double* norms, int* active, int B, double thresh, int* count)
{
    GRID_STRIDE(i, B)
    {
        double sum = 0.0;
        for (int q = 0; q < P; ++q) sum += part[static_cast<size_t>(i) * P + q];
        const double nr = sqrt(sum);
        norms[i] = nr;
        const int a = nr > thresh ? 1 : 0;
        active[i] = a;
        if (a) atomicAdd(count, 1);
    }
}

// Control of a device-side refinement loop (the body of a conditional WHILE
// node of a round graph), the same decisions as the host loop of the
// converged form: at iteration it (iter[0]) with cnt samples above the
// threshold, stop when cnt = 0; when it has reached max_iter, stop and record
// NOT_CONVERGED; else run the body once more. iter[MLQMC_MAX_LEVELS] keeps the
// largest iteration reached. The count is cleared for the next pass.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, int* count, int* iter, int max_iter, int* status)
{
    const int cnt = *count;
    *count = 0;
    const int it = iter[0];
    if (it > iter[MLQMC_MAX_LEVELS]) iter[MLQMC_MAX_LEVELS] = it;
    unsigned go = 0;
    if (cnt > 0) {
        if (it >= max_iter) {
            atomicOr(status, kStatusNotConverged);
        } else {
            go = 1;
            iter[0] = it + 1;
        }
    }
    cudaGraphSetConditional(h, go);
}

// Zero n 16-byte words (the correction of a level inside a loop body, where a
// graph takes kernel nodes).
__global__ void k_zero16(uint4* p, size_t n)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        p[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Team index and count of a flat grid: one CTA or one warp per sample.
template <typename TM>
__device__ __forceinline__ int team_index()
{
    if constexpr (std::is_same<TM, WarpTeam>::value) return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    else return blockIdx.x;
}

template <typename TM>
__device__ __forceinline__ int team_count()
{
    if constexpr (std::is_same<TM, WarpTeam>::value) return gridDim.x * (blockDim.x >> 5);
    else return gridDim.x;
}

// F_t of samples 0..B-1: one CTA per sample on large levels, one warp per
// sample on small ones (TM), the sum in a fixed order either way.
// UPD (mixed forms, one refinement step per level): the step's last update
// u64 += e (e the FP32 correction in u), the FP32 copy of u64 and the sum run
// in one pass over each thread's cell pairs, so u64 is read once; the new
// u64 is stored only when something reads it later (keep64: the centre QoI,
// the solution output), else only its FP32 copy and the sum leave the pass.
template <typename T, bool U64, typename TM, bool UPD = false>
__global__ void __launch_bounds__(256) kb_qoi(FmgArgs A, int t, int B, int keep64)
{
    static_assert(!UPD || (U64 && sizeof(T) == 4), "the fused update is the mixed forms' refinement step");
    __shared__ double red[48];
    const TM tm;
    for (int i = team_index<TM>(); i < B; i += team_count<TM>()) {
        double v;
        if constexpr (UPD) {
            double2* u64 = reinterpret_cast<double2*>(at<double>(A.lv[t].u64, i));
            float2* u = reinterpret_cast<float2*>(at<float>(A.lv[t].u, i));
            const int n = A.lv[t].n;
            const int np = n * n / 2, sz = tm.size();
            double acc = 0.0;
            // four pairs per round, all loads first (the stores could alias the
            // next loads as far as the compiler knows); cells summed in p order
            constexpr int U = 4;
            int p = tm.rank();
            for (; p + (U - 1) * sz < np; p += U * sz) {
                double2 w[U];
                float2 d[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    w[k] = u64[p + k * sz];
                    d[k] = u[p + k * sz];  // the correction e, replaced by the FP32 copy of u64
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const double2 r = make_double2(w[k].x + widen(d[k].x), w[k].y + widen(d[k].y));
                    if (keep64) u64[p + k * sz] = r;
                    u[p + k * sz] = make_float2(narrow(r.x), narrow(r.y));
                    acc += r.x;
                    acc += r.y;
                }
            }
            for (; p < np; p += sz) {
                const double2 w = u64[p];
                const float2 d = u[p];
                const double2 r = make_double2(w.x + widen(d.x), w.y + widen(d.y));
                if (keep64) u64[p] = r;
                u[p] = make_float2(narrow(r.x), narrow(r.y));
                acc += r.x;
                acc += r.y;
            }
            if (A.qoi == MLQMC_QOI_MEAN) {
                v = team_sum(tm, acc, red) / (static_cast<double>(n) * n);
            } else {
                tm.sync();
                v = qoi(tm, at<double>(A.lv[t].u64, i), n, A.qoi, red);
            }
        } else {
            if constexpr (U64) v = qoi(tm, at<double>(A.lv[t].u64, i), A.lv[t].n, A.qoi, red);
            else v = qoi(tm, at<T>(A.lv[t].u, i), A.lv[t].n, A.qoi, red);
        }
        if (tm.leader()) A.F[static_cast<size_t>(i) * A.n_levels + t] = v;
        if constexpr (U64 && sizeof(T) == 4 && !UPD) {
            // mixed forms: FP32 copy of the level's solution for the next FMG interpolation
            const double2* u64 = reinterpret_cast<const double2*>(at<double>(A.lv[t].u64, i));
            float2* u = reinterpret_cast<float2*>(at<float>(A.lv[t].u, i));
            const int nn2 = A.lv[t].n * A.lv[t].n / 2;
            for (int p = tm.rank(); p < nn2; p += tm.size()) {
                const double2 w = u64[p];
                u[p] = make_float2(narrow(w.x), narrow(w.y));
            }
        }
    }
}

// F_t on large levels in chunks, so that a few large samples still fill the
// GPU: CTA (i, q) of the B x P grid takes the cell pairs [q csz, (q+1) csz)
// of sample i with the per-cell work of kb_qoi (UPD: u64 += e, the FP32 copy
// of u64, the sum; U64 with FP32 work arrays: the FP32 copy and the sum;
// else the sum) and writes its partial sum; kb_qoi_final adds each sample's
// partials in order.
template <typename T, bool U64, bool UPD>
__global__ void __launch_bounds__(256) kb_qoi_part(FmgArgs A, int t, int B, int P, double* part, int keep64,
                                                   int interp32)
{
    static_assert(!UPD || (U64 && sizeof(T) == 4), "the fused update is the mixed forms' refinement step");
    __shared__ double red[48];
    const int n = A.lv[t].n;
    const int np = n * n / 2;  // cell pairs (n even)
    const int csz = (np + P - 1) / P;
    constexpr int kT = 256;
    for (int w = blockIdx.x; w < B * P; w += gridDim.x) {  // uniform per CTA: every thread reaches block_sum
        const int i = w / P, q = w - i * P;
        const int p0 = q * csz, p1 = min(np, p0 + csz);
        double acc = 0.0;
        if (UPD && interp32) {
            // the interpolant U in FP32 (the level's field array): U + e exactly
            // as the TwoSum pair, its high part the FP32 copy
            PairSum ps;
            const float2* kf = reinterpret_cast<const float2*>(at<float>(A.lv[t].k, i));
            float2* u = reinterpret_cast<float2*>(at<float>(A.lv[t].u, i));
            constexpr int U = 4;
            int p = p0 + static_cast<int>(threadIdx.x);
            for (; p + (U - 1) * kT < p1; p += U * kT) {
                float2 w[U], d[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    w[k] = kf[p + k * kT];
                    d[k] = u[p + k * kT];
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    float2 h, lo;
                    two_sum32(w[k].x, d[k].x, h.x, lo.x);
                    two_sum32(w[k].y, d[k].y, h.y, lo.y);
                    u[p + k * kT] = h;
                    ps.add(h.x, lo.x);
                    ps.add(h.y, lo.y);
                }
            }
            for (; p < p1; p += kT) {
                const float2 w = kf[p], d = u[p];
                float2 h, lo;
                two_sum32(w.x, d.x, h.x, lo.x);
                two_sum32(w.y, d.y, h.y, lo.y);
                u[p] = h;
                ps.add(h.x, lo.x);
                ps.add(h.y, lo.y);
            }
            acc = ps.value();
        } else if constexpr (U64) {
            // mixed forms: the sum from the FP32 copy and its remainder (PairSum)
            PairSum ps;
            double2* u64 = reinterpret_cast<double2*>(at<double>(A.lv[t].u64, i));
            float2* u = reinterpret_cast<float2*>(at<float>(A.lv[t].u, i));
            constexpr int U = 4;
            int p = p0 + static_cast<int>(threadIdx.x);
            for (; p + (U - 1) * kT < p1; p += U * kT) {
                double2 r[U];
                float2 d[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    r[k] = u64[p + k * kT];
                    if constexpr (UPD) d[k] = u[p + k * kT];
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    if constexpr (UPD) {
                        float2 h, lo;
                        double2 rr = make_double2(0.0, 0.0);
                        update_pair(r[k].x, d[k].x, keep64, h.x, lo.x, rr.x);
                        update_pair(r[k].y, d[k].y, keep64, h.y, lo.y, rr.y);
                        if (keep64) u64[p + k * kT] = rr;
                        u[p + k * kT] = h;
                        ps.add(h.x, lo.x);
                        ps.add(h.y, lo.y);
                    } else if constexpr (sizeof(T) == 4) {
                        const float2 h = make_float2(narrow(r[k].x), narrow(r[k].y));
                        u[p + k * kT] = h;
                        ps.add(h.x, narrow_rest(r[k].x, h.x));
                        ps.add(h.y, narrow_rest(r[k].y, h.y));
                    } else {
                        acc += r[k].x;
                        acc += r[k].y;
                    }
                }
            }
            for (; p < p1; p += kT) {
                const double2 r = u64[p];
                if constexpr (UPD) {
                    const float2 d = u[p];
                    float2 h, lo;
                    double2 rr = make_double2(0.0, 0.0);
                    update_pair(r.x, d.x, keep64, h.x, lo.x, rr.x);
                    update_pair(r.y, d.y, keep64, h.y, lo.y, rr.y);
                    if (keep64) u64[p] = rr;
                    u[p] = h;
                    ps.add(h.x, lo.x);
                    ps.add(h.y, lo.y);
                } else if constexpr (sizeof(T) == 4) {
                    const float2 h = make_float2(narrow(r.x), narrow(r.y));
                    u[p] = h;
                    ps.add(h.x, narrow_rest(r.x, h.x));
                    ps.add(h.y, narrow_rest(r.y, h.y));
                } else {
                    acc += r.x;
                    acc += r.y;
                }
            }
            if constexpr (sizeof(T) == 4) acc = ps.value();
        } else {
            const T* u = at<T>(A.lv[t].u, i);
            for (int p = p0 + static_cast<int>(threadIdx.x); p < p1; p += kT) {
                acc += static_cast<double>(u[2 * p]);
                acc += static_cast<double>(u[2 * p + 1]);
            }
        }
        const double sum = block_sum(acc, red);
        if (threadIdx.x == 0) part[w] = sum;
    }
}

// F_t of samples 0..B-1 from the chunk sums (mean of u, partials added in
// order) or from the four centre cells (centre QoI).
template <typename T, bool U64>
__global__ void kb_qoi_final(FmgArgs A, int t, int B, int P, const double* __restrict__ part)
{
    const int n = A.lv[t].n;
    GRID_STRIDE(i, B)
    {
        double v;
        if (A.qoi == MLQMC_QOI_MEAN) {
            double sum = 0.0;
            for (int q = 0; q < P; ++q) sum += part[static_cast<size_t>(i) * P + q];
            v = sum / (static_cast<double>(n) * n);
        } else {
            const int m = n / 2;
            const int c[4] = {(m - 1) * n + (m - 1), (m - 1) * n + m, m * n + (m - 1), m * n + m};
            double s4 = 0.0;
            for (int k = 0; k < 4; ++k) {
                if constexpr (U64) s4 += at<double>(A.lv[t].u64, i)[c[k]];
                else s4 += static_cast<double>(at<T>(A.lv[t].u, i)[c[k]]);
            }
            v = 0.25 * s4;
        }
        A.F[static_cast<size_t>(i) * A.n_levels + t] = v;
    }
}

// k of level t (samples 0..B-1) widened to FP64, by canon (introspection).
template <typename T>
__global__ void kb_k_out(FmgArgs A, int t, int B, double* out)
{
    const int n = A.lv[t].n;
    const uint32_t per = static_cast<uint32_t>(n) * static_cast<uint32_t>(n);
    GRID_STRIDE(idx, B * per)
    {
        const int i = static_cast<int>(A.lv[t].by_nn.div(idx));
        const int p = static_cast<int>(idx - i * per);
        out[static_cast<size_t>(A.samples[i].canon) * per + p] = static_cast<double>(at<T>(A.lv[t].k, i)[p]);
    }
}

// Solution of level t of sample 0 widened to FP64 (introspection).
template <typename T, bool U64>
__global__ void kb_u_out(FmgArgs A, int t, double* out)
{
    const int n = A.lv[t].n;
    GRID_STRIDE(p, static_cast<uint32_t>(n) * static_cast<uint32_t>(n))
    {
        if constexpr (U64) out[p] = at<double>(A.lv[t].u64, 0)[p];
        else out[p] = static_cast<double>(at<T>(A.lv[t].u, 0)[p]);
    }
}

// Deterministic reuse sums per (level t, shift r): one block each, rank order.
__global__ void k_sums(const SampleDesc* __restrict__ smp, int n, const double* __restrict__ F, int n_levels, int R,
                       int reuse, double* __restrict__ sums)
{
    __shared__ double red[48];
    const int t = blockIdx.x / R;
    const int r = blockIdx.x - t * R;
    double a = 0.0, a2 = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const SampleDesc d = smp[q];
        if (d.r == r && (reuse ? d.level >= t : d.level == t)) {
            const double* Fq = F + static_cast<size_t>(q) * n_levels;
            const double v = Fq[t] - (t > 0 ? Fq[t - 1] : 0.0);
            a += v;
            a2 += v * v;
        }
    }
    a = block_sum(a, red);
    a2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        sums[(static_cast<size_t>(t) * R + r) * 2 + 0] += a;
        sums[(static_cast<size_t>(t) * R + r) * 2 + 1] += a2;
    }
}

// Per-sample F_0..F_level (zeros above) in work order.
__global__ void k_fout(const SampleDesc* __restrict__ smp, int n, const double* __restrict__ F, int n_levels,
                       double* __restrict__ out)
{
    GRID_STRIDE(idx, static_cast<uint32_t>(n) * static_cast<uint32_t>(n_levels))
    {
        const int q = static_cast<int>(idx / n_levels);
        const int t = static_cast<int>(idx - static_cast<int64_t>(q) * n_levels);
        const SampleDesc d = smp[q];
        out[static_cast<size_t>(d.gidx) * n_levels + t] = t <= d.level ? F[static_cast<size_t>(q) * n_levels + t] : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
inline bool ok(cudaError_t e) { return e == cudaSuccess; }

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool is_mixed(const mlqmc_problem& p) { return p.precision != MLQMC_FP64; }

size_t elem_size(const mlqmc_problem& p) { return is_mixed(p) ? sizeof(float) : sizeof(double); }

// Bytes per sample of each pooled array of level t.
void level_strides(const mlqmc_problem& p, int Ka, int t, size_t st[kPoolArrs])
{
    const size_t n = static_cast<size_t>(p.coarse_cells) << t;
    const size_t es = elem_size(p);
    st[kU] = align256(es * n * n);
    st[kBc] = align256(es * n * n);
    st[kKx] = align256(es * n * kx_pitch(static_cast<int>(n)));
    st[kKy] = align256(es * n * (n + 1));
    st[kIdiag] = align256(es * n * n);
    st[kK] = align256(es * n * n);
    st[kG] = align256(es * static_cast<size_t>(std::max(Ka, 1)) * n);
    st[kU64] = (is_mixed(p) || p.refine_rtol > 0.0) ? align256(8 * n * n) : 0;
    st[kU2] = t > 0 ? align256(es * n * n) : 0;
}

// Most elements one sample of level t has in a flat kernel loop (faces, cells, KL partial sums).
uint64_t level_elems_per_sample(const mlqmc_problem& p, int Ka, int t)
{
    const uint64_t n = static_cast<uint64_t>(p.coarse_cells) << t;
    return std::max<uint64_t>(n * (n + 1), static_cast<uint64_t>(std::max(Ka, 1)) * n);
}

size_t level_bytes_per_sample(const mlqmc_problem& p, int Ka, int t)
{
    size_t st[kPoolArrs];
    level_strides(p, Ka, t, st);
    size_t b = 0;
    for (int a = 0; a < kPoolArrs; ++a) b += st[a];
    return b;
}

// Grow the pool of level t to hold at least `need` samples.
mlqmc_status ensure_pool(mlqmc_ctx* c, int t, int64_t need)
{
    LevelPool& P = c->pools[t];
    if (need <= P.cap) return MLQMC_OK;
    size_t st[kPoolArrs];
    level_strides(c->p, c->Ka, t, st);
    // Algorithm 1 doubles a level's count round by round, and each growth
    // waits for the device and reallocates: small pools grow fourfold, so
    // that two doublings fit, large ones by half
    const size_t per = level_bytes_per_sample(c->p, c->Ka, t);
    const bool small = per * static_cast<size_t>(4 * std::max<int64_t>(P.cap, need)) <= (size_t(256) << 20);
    const int64_t cap = std::max<int64_t>(need, small ? 4 * P.cap : P.cap + P.cap / 2);
    size_t off = 0, offs[kPoolArrs];
    for (int a = 0; a < kPoolArrs; ++a) {
        offs[a] = off;
        off += st[a] * static_cast<size_t>(cap);
    }
    if (P.mem) {
        cudaDeviceSynchronize();
        cudaFree(P.mem);
        P.mem = nullptr;
        P.cap = 0;
    }
    ++c->pool_epoch;
    if (!ok(cudaMalloc(&P.mem, std::max<size_t>(off, 256)))) {
        cudaGetLastError();
        P.mem = nullptr;
        return MLQMC_ERR_OOM;
    }
    P.cap = cap;
    for (int a = 0; a < kPoolArrs; ++a) {
        P.off[a] = offs[a];
        P.stride[a] = st[a];
    }
    return MLQMC_OK;
}

FmgArgs base_args(mlqmc_ctx* c)
{
    FmgArgs A;
    std::memset(&A, 0, sizeof(A));
    A.samples = c->d_samples;
    A.Y = c->d_Y;
    A.c32 = c->d_c32;
    A.s = c->p.n_modes;
    A.n0 = c->p.coarse_cells;
    A.n_levels = c->p.n_levels;
    A.qoi = c->p.qoi;
    A.mu0 = c->p.mu0;
    A.nu1 = c->p.nu1;
    A.nu2 = c->p.nu2;
    A.rtol = c->p.refine_rtol;
    A.max_iter = c->p.refine_max_iter;
    A.Ka = c->Ka;
    A.psi = is_mixed(c->p) ? static_cast<const void*>(c->d_psi32) : static_cast<const void*>(c->d_psi);
    for (int t = 0; t < c->p.n_levels; ++t) A.psi_off[t] = c->psi_off[t];
    A.grp_start = c->d_grp_start;
    A.grp_b = c->d_grp_b;
    A.grp_m = c->d_grp_m;
    A.grp_sqrt = c->d_grp_sqrt;
    for (int t = 0; t < c->p.n_levels; ++t) {
        const LevelPool& P = c->pools[t];
        LevelDesc& d = A.lv[t];
        d.n = c->p.coarse_cells << t;
        set_divisors(d, c->Ka);
        ArrDesc* arr[kPoolArrs] = {&d.u, &d.bc, &d.kx, &d.ky, &d.idiag, &d.k, &d.G, &d.u64, &d.u2};
        for (int a = 0; a < kPoolArrs; ++a) {
            arr[a]->base = P.mem ? P.mem + P.off[a] : nullptr;
            arr[a]->stride = P.stride[a];
        }
    }
    A.chol.base = reinterpret_cast<unsigned char*>(c->d_chol);
    A.chol.stride = static_cast<size_t>(c->max_samples);  // interleaved: entry q of sample i at q * max_samples + i
    A.chol32 = c->d_chol32;
    A.F = c->d_F;
    A.queue = c->d_queue;
    A.status = c->d_status;
    A.norms = c->d_norms;
    A.refine = (is_mixed(c->p) || c->p.refine_rtol > 0.0) ? 1 : 0;
    return A;
}

cudaEvent_t take_event(mlqmc_ctx* c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Algorithmic work of one launch: the bytes it must move when every array it
// touches is read or written once, and its arithmetic by precision.
struct Work {
    double bytes = 0.0, f64 = 0.0, f32 = 0.0, ftc = 0.0;
};

template <typename T>
Work work_of(double bytes, double flops)
{
    Work w;
    w.bytes = bytes;
    if (sizeof(T) == 8) w.f64 = flops;
    else w.f32 = flops;
    return w;
}

// Brackets one launch with events when profiling is on and adds its work.
// nk: kernels launched inside the bracket.
struct Timed {
    mlqmc_ctx* c;
    int kind;
    int level;
    cudaStream_t st;
    int nk;
    cudaEvent_t a = nullptr;
    Timed(mlqmc_ctx* c_, int kind_, cudaStream_t st_, const Work& w = Work(), int nk_ = 1)
        : c(c_), kind(kind_), level(c_->prof_level), st(st_), nk(nk_)
    {
        if (c->profiling) {
            a = take_event(c);
            record(a);
            ProfCell& pc = c->prof[kind][level];
            pc.bytes += w.bytes;
            pc.f64 += w.f64;
            pc.f32 += w.f32;
            pc.ftc += w.ftc;
        }
    }
    ~Timed()
    {
        c->launches += nk;
        if (!a) return;
        cudaEvent_t b = take_event(c);
        record(b);
        c->marks.push_back({kind, level, nk, a, b});
    }
    // inside a stream capture the record must become an event-record node of
    // the graph (external), so that the host can time every replay
    void record(cudaEvent_t e) const
    {
        if (c->graph.capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    }
};

// The grid level that the brackets of the enclosing scope belong to.
struct LevelTag {
    mlqmc_ctx* c;
    int prev;
    LevelTag(mlqmc_ctx* c_, int t) : c(c_), prev(c_->prof_level) { c->prof_level = t; }
    ~LevelTag() { c->prof_level = prev; }
};

// Cells and faces of one direction on level t.
double cells_of(const mlqmc_ctx* c, int t)
{
    const double n = static_cast<double>(c->p.coarse_cells << t);
    return n * n;
}

double faces_of(const mlqmc_ctx* c, int t)
{
    const double n = static_cast<double>(c->p.coarse_cells << t);
    return n * (n + 1.0);
}

int grid_for(mlqmc_ctx* c, int64_t work, int threads = 256)
{
    const int64_t want = (work + threads - 1) / threads;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(c->sm_count) * 32)));
}

// Chunks per sample of the large-level QoI pass (about 65536 cells each).
int qoi_chunks(const mlqmc_ctx* c, int t)
{
    const int64_t n = c->p.coarse_cells << t;
    return static_cast<int>(std::max<int64_t>(1, n * n / 65536));
}

// Room for the QoI partial sums of Bt[t] samples on every level t <= Lmax
// (grown outside any capture; a new buffer invalidates captured graphs).
mlqmc_status ensure_qpart(mlqmc_ctx* c, const int* Bt, int Lmax)
{
    int64_t need = 0;
    for (int t = 0; t <= Lmax; ++t) need = std::max<int64_t>(need, static_cast<int64_t>(Bt[t]) * qoi_chunks(c, t));
    if (need <= c->qpart_cap) return MLQMC_OK;
    cudaDeviceSynchronize();
    cudaFree(c->d_qpart);
    c->d_qpart = nullptr;
    c->qpart_cap = 0;
    ++c->pool_epoch;
    if (!ok(cudaMalloc(&c->d_qpart, sizeof(double) * static_cast<size_t>(need)))) return MLQMC_ERR_OOM;
    c->qpart_cap = need;
    return MLQMC_OK;
}

mlqmc_status last_error()
{
    return ok(cudaGetLastError()) ? MLQMC_OK : MLQMC_ERR_CUDA;
}

// Calls with fewer level-0 samples than this take kb_level0_split.
constexpr int kLevel0SplitBelow = 16384;

// Level-0 factor, exact solve and F_0 of samples 0..B-1.
mlqmc_status launch_level0(mlqmc_ctx* c, const FmgArgs& A, int B, cudaStream_t st)
{
    LevelTag lt(c, 0);
    // per sample: faces in, band factor (n0 + 1 entries per row) and solutions out;
    // banded Cholesky N0 n0^2 and two triangular solves 4 N0 n0 FP64 FLOPs
    const double N0 = cells_of(c, 0), n0 = c->p.coarse_cells, es = is_mixed(c->p) ? 4.0 : 8.0;
    Work w;
    w.bytes = B * (es * (2.0 * faces_of(c, 0)) + 8.0 * N0 * (n0 + 1.0) + (is_mixed(c->p) ? 4.0 * N0 * (n0 + 1.0) : 0.0) +
                   (8.0 + es) * N0 + 8.0);
    w.f64 = B * (N0 * n0 * n0 + 4.0 * N0 * n0);
    Timed tm(c, kProfSmall, st, w);
    // n0 = 8: one wave of resident CTAs (shared memory allows five per SM),
    // each looping over its samples, so that all of them are placed at once
    // and the other stream's kernels are not queued behind a second wave
    int per_sm = 8;
    if (c->p.coarse_cells == 8) {
        const bool mx = is_mixed(c->p);
        if (!ok(mx ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_level0_fixed<float, true, 8>, 64,
                                                                  level0_smem<8>())
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_level0_fixed<double, false, 8>, 64,
                                                                  level0_smem<8>())))
            return MLQMC_ERR_CUDA;
        per_sm = std::max(1, per_sm);
    }
    const int g64 = std::max(1, std::min((B + 63) / 64, c->sm_count * per_sm));
    // few samples: one thread per sample would leave most SM sub-partitions
    // idle, each warp's FP64 chain alone setting the time; split every step
    // of a group of 32 samples over the warps of a CTA instead (same results)
    const int g32 = (B + 31) / 32;
    if (B < kLevel0SplitBelow && (c->p.coarse_cells == 8 || c->p.coarse_cells == 4)) {
        if (c->p.coarse_cells == 8) {
            if (is_mixed(c->p)) kb_level0_split<float, true, 8><<<g32, 32 * 10, 0, st>>>(A, B);
            else kb_level0_split<double, false, 8><<<g32, 32 * 10, 0, st>>>(A, B);
        } else {
            if (is_mixed(c->p)) kb_level0_split<float, true, 4><<<g32, 32 * 6, 0, st>>>(A, B);
            else kb_level0_split<double, false, 4><<<g32, 32 * 6, 0, st>>>(A, B);
        }
    } else if (c->p.coarse_cells == 8) {
        if (is_mixed(c->p)) kb_level0_fixed<float, true, 8><<<g64, 64, level0_smem<8>(), st>>>(A, B);
        else kb_level0_fixed<double, false, 8><<<g64, 64, level0_smem<8>(), st>>>(A, B);
    } else if (c->p.coarse_cells == 4) {
        if (is_mixed(c->p)) kb_level0_fixed<float, true, 4><<<g64, 64, level0_smem<4>(), st>>>(A, B);
        else kb_level0_fixed<double, false, 4><<<g64, 64, level0_smem<4>(), st>>>(A, B);
    } else if (is_mixed(c->p)) {
        kb_level0<float, true><<<grid_for(c, B, 128), 128, 0, st>>>(A, B);
    } else {
        kb_level0<double, false><<<grid_for(c, B, 128), 128, 0, st>>>(A, B);
    }
    return last_error();
}

template <typename T>
void launch_coarse(mlqmc_ctx* c, const FmgArgs& A, int B, cudaStream_t st)
{
    if (c->p.coarse_cells == 8) {
        kb_coarse_fixed<T, 8><<<std::max(1, std::min((B + 63) / 64, c->sm_count * 32)), 64, 0, st>>>(A, B);
        return;
    }
    if (c->p.coarse_cells == 4) {
        kb_coarse_fixed<T, 4><<<std::max(1, std::min((B + 63) / 64, c->sm_count * 32)), 64, 0, st>>>(A, B);
        return;
    }
    const size_t N0 = static_cast<size_t>(c->p.coarse_cells) * c->p.coarse_cells;
    const size_t smem = N0 * 64 * sizeof(T);
    if (smem <= 48 * 1024) kb_coarse<T, true><<<grid_for(c, B, 64), 64, smem, st>>>(A, B);
    else kb_coarse<T, false><<<grid_for(c, B, 64), 64, 0, st>>>(A, B);
}

mlqmc_status launch_points(mlqmc_ctx* c, const SampleDesc* d_s, int count, double* Y, uint64_t* bits, cudaStream_t st)
{
    const int64_t total = static_cast<int64_t>(count) * c->p.n_modes;
    Timed tm(c, kProfPoints, st, work_of<double>(8.0 * total + sizeof(SampleDesc) * count, 0.0));
    k_points<<<grid_for(c, total), 256, 0, st>>>(d_s, count, c->p.n_modes, c->p.sampler, c->p.seed, c->d_z,
                                                 c->d_shift, c->p.n_shifts, Y, bits, is_mixed(c->p) ? 1 : 0);
    return last_error();
}

// Smoother of level t's sweeps for a call with B samples on the level (the
// autotuner's batch-size schedule).
int smoother_for(const mlqmc_ctx* c, int t, int B)
{
    return B < kSmallBatch ? c->smoother_small[t] : c->smoother[t];
}

// Samples per tile of the tensor-core KL of level t for B samples.
int kl_nt_for(const mlqmc_ctx* c, int t, int B)
{
    return c->kl_nt[t][B < kSmallBatch ? 0 : 1];
}

// Whether smoother kind k can run level t in the context's form (FP64: kb_gs,
// the whole-sample smoother and the plain tiles; the TMA-tiled and wavefront
// ones are FP32 only).
bool smoother_fits(const mlqmc_ctx* c, int k, int t)
{
    const int n = c->p.coarse_cells << t;
    if (!is_mixed(c->p) && k != MLQMC_SMOOTHER_GS && k != MLQMC_SMOOTHER_WHOLE && k != MLQMC_SMOOTHER_TILE)
        return false;
    switch (k) {
    case MLQMC_SMOOTHER_STREAM: return mlqmc_stream::supported(n);
    case MLQMC_SMOOTHER_TMA: return mlqmc_tma::supported(n);
    case MLQMC_SMOOTHER_WHOLE: return mlqmc_whole::supported(n, !is_mixed(c->p));
    case MLQMC_SMOOTHER_TILE: return n == 8 || n == 16 || (n >= 32 && n % 32 == 0);
    default: return true;
    }
}

// True when level t's field comes from the tensor-core contraction.
bool uses_tc(const mlqmc_ctx* c, int t)
{
    return c->kl_tc && c->d_psi_tc[t] != nullptr;
}

enum class SynthPart { all, field, faces };

// Batched KL field and faces of level t for samples 0..B-1. The field comes
// from the tensor-core contraction (mixed forms, every level)
// or from the separable SIMT sum; the C operand must already be built.
// part: the tensor-core field alone, or the faces alone (after it).
template <typename T>
mlqmc_status synth_batched(mlqmc_ctx* c, const FmgArgs& A, int t, int B, cudaStream_t st,
                           SynthPart part = SynthPart::all)
{
    LevelTag lt(c, t);
    const int64_t n = c->p.coarse_cells << t;
    if constexpr (sizeof(T) == 4) {
        if (uses_tc(c, t) && part != SynthPart::faces) {
            const LevelPool& P = c->pools[t];
            float* k = reinterpret_cast<float*>(P.mem + P.off[kK]);
            const double M = static_cast<double>(n * n);
            const double K = static_cast<double>(mlqmc_kl::row_bytes(c->kl_variant, c->p.n_modes)) / 4.0;
            Work w;
            w.bytes = 4.0 * (M * B + M * K + B * K);  // k out, Psi and C in
            w.ftc = 2.0 * M * c->p.n_modes * B;
            Timed tm(c, kProfKlTc, st, w);
            if (!mlqmc_kl::launch(c->kl_variant, c->kl_maps[t], static_cast<int>(n * n), B, c->p.n_modes, k,
                                  P.stride[kK] / sizeof(float), c->d_status, st, kl_nt_for(c, t, B)))
                return MLQMC_ERR_CUDA;
        }
    }
    if (part == SynthPart::faces) {
    } else if (c->matern && (!uses_tc(c, t) || sizeof(T) != 4)) {
        const double M = static_cast<double>(n * n), sm = c->p.n_modes;
        Timed tm(c, kProfSynth, st,
                 work_of<T>(8.0 * M * sm * std::ceil(B / static_cast<double>(kDenseG)) + sizeof(T) * M * B,
                            2.0 * M * sm * B));
        const dim3 grid(static_cast<unsigned>((n * n + 255) / 256), static_cast<unsigned>((B + kDenseG - 1) / kDenseG));
        kb_synth_dense<T><<<grid, 256, 0, st>>>(A, t, B, c->d_psi_dense + c->dense_off[t], c->p.n_modes,
                                               c->d_sqrt_theta);
    } else if (!uses_tc(c, t) || sizeof(T) != 4) {
        const double M = static_cast<double>(n * n), Ka = c->Ka, sm = c->p.n_modes;
        if constexpr (sizeof(T) == 4) {
            if (!c->c32_ready) {
                Timed tm(c, kProfSynth, st, work_of<double>(B * 12.0 * sm, B * sm));
                k_coef32<<<grid_for(c, static_cast<int64_t>(B) * c->p.n_modes), 256, 0, st>>>(A, B, c->d_sqrt_theta,
                                                                                           c->d_c32);
            }
        }
        {
            Timed tm(c, kProfSynth, st, work_of<T>(B * (sizeof(T) * sm + sizeof(T) * Ka * n), B * 2.0 * sm * n));
            kb_synth_G<T><<<grid_for(c, B * c->Ka * n), 256, 0, st>>>(A, t, B);
        }
        {
            Timed tm(c, kProfSynth, st, work_of<T>(B * sizeof(T) * (Ka * n + M), B * 2.0 * Ka * M));
            kb_synth_z<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
        }
    }
    if (part == SynthPart::field) return last_error();
    const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
    {
        Timed tm(c, kProfSynth, st, work_of<T>(B * es * (Mc + 2.0 * Fc), B * 6.0 * Fc));
        if (sizeof(T) == 4 && n % 4 == 0) kb_faces4<<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B);
        else kb_faces<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
    }
    if (t > 0 && (sizeof(T) == 8 || smoother_for(c, t, B) <= MLQMC_SMOOTHER_TILE)) {  // 1/D: FP64 sweeps, tiles
        Timed tm(c, kProfSynth, st, work_of<T>(B * es * (2.0 * Fc + Mc), B * 5.0 * Mc));
        kb_idiag<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
    }
    return last_error();
}

// C operand of the tensor-core contraction for samples 0..count-1 (normals in rank order).
mlqmc_status build_c(mlqmc_ctx* c, int count, cudaStream_t st)
{
    if (!c->kl_tc) return MLQMC_OK;
    Timed tm(c, kProfKlTc, st,
             work_of<float>(count * (8.0 * c->p.n_modes + mlqmc_kl::row_bytes(c->kl_variant, c->p.n_modes)), 0.0));
    return mlqmc_kl::build_c(c->kl_variant, c->d_Y, nullptr, count, c->p.n_modes, c->d_sqrt_theta, c->d_C, st)
               ? MLQMC_OK
                                                                                                : MLQMC_ERR_CUDA;
}

mlqmc_status zero_u(mlqmc_ctx* c, int t, int B, cudaStream_t st)
{
    LevelTag lt(c, t);
    const LevelPool& P = c->pools[t];
    const size_t bytes = P.stride[kU] * static_cast<size_t>(B);  // strides are multiples of 256 bytes
    if (c->graph.in_body) {
        Timed tm(c, kProfTransfer, st, work_of<double>(static_cast<double>(bytes), 0.0));
        k_zero16<<<grid_for(c, static_cast<int64_t>(bytes / 16)), 256, 0, st>>>(
            reinterpret_cast<uint4*>(P.mem + P.off[kU]), bytes / 16);
        return last_error();
    }
    return ok(cudaMemsetAsync(P.mem + P.off[kU], 0, bytes, st)) ? MLQMC_OK : MLQMC_ERR_CUDA;
}

// V-cycle on level t_top (>= 1) for samples 0..B-1: batched sweeps and
// transfers down to level 1, the coarse solve on level 0, and back up. ones:
// the top right-hand side is 1 (FP64 form), else bc of t_top (mixed correction).
// Swap the roles of u and u2 on level t (after a ping-pong smoothing launch).
void swap_u(mlqmc_ctx* c, FmgArgs& A, int t)
{
    std::swap(c->pools[t].off[kU], c->pools[t].off[kU2]);
    std::swap(A.lv[t].u, A.lv[t].u2);
}

template <typename T, int TILE, int NS>
constexpr size_t tile_smem()
{
    constexpr int SU = TILE + 2 * TileHalo<T, NS>::H;
    return sizeof(T) * (3 * SU * SU + 2 * (SU + 1) * SU);
}

template <typename T, int TILE, int NS>
void launch_tile(mlqmc_ctx* c, const FmgArgs& A, int t, int B, int ones, int first, bool pro, cudaStream_t st)
{
    const int64_t n = c->p.coarse_cells << t;
    const int64_t tiles = B * (n / TILE) * (n / TILE);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tiles, c->sm_count * 16)));
    constexpr size_t smem = tile_smem<T, TILE, NS>();
    if (pro) kb_rbgs_tile<T, TILE, NS, true><<<grid, 256, smem, st>>>(A, t, B, ones, first);
    else kb_rbgs_tile<T, TILE, NS, false><<<grid, 256, smem, st>>>(A, t, B, ones, first);
}

template <typename T, int TILE, int NS>
bool tile_attr()
{
    const int b = static_cast<int>(tile_smem<T, TILE, NS>());
    return cudaFuncSetAttribute(kb_rbgs_tile<T, TILE, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kb_rbgs_tile<T, TILE, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) ==
               cudaSuccess;
}

// FP32 tiles take two sweeps per launch (memory-bound, the halo work is
// cheap); FP64 tiles one (FP64 arithmetic is the scarce resource on GB300:
// a second sweep would add 21 % halo updates to save 24 of 48 bytes per cell).
template <typename T>
constexpr int tile_sweeps()
{
    return sizeof(T) == 8 ? 1 : 2;
}

template <int TILE>
bool tile_attrs()
{
    return tile_attr<float, TILE, 2>() && tile_attr<float, TILE, 1>() && tile_attr<double, TILE, 1>();
}

// nsweeps full red-black sweeps of level t (first: colour of the first half
// sweep), on tiles of 8, 16 or 32 cells where the level's smoother is the
// plain-tile one, else (FP64 form, sides that are not such a multiple) two
// kb_gs launches per sweep.
template <typename T>
int tile_side(const mlqmc_ctx* c, int t, int B)
{
    const int64_t n = c->p.coarse_cells << t;
    if (smoother_for(c, t, B) != MLQMC_SMOOTHER_TILE) return 0;
    return n >= 32 && n % 32 == 0 ? 32 : (n == 16 ? 16 : (n == 8 ? 8 : 0));
}

// pro: add the coarse-grid correction P e first (post-smoothing).
template <typename T>
void smooth(mlqmc_ctx* c, FmgArgs& A, int t, int B, int nsweeps, int first, int ones, bool pro, cudaStream_t st)
{
    LevelTag lt(c, t);
    const int64_t n = c->p.coarse_cells << t;
    const int tile = tile_side<T>(c, t, B);
    const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
    const Work pro_work = work_of<T>(B * es * (0.25 * Mc + 2.0 * Mc), B * 8.0 * Mc);
    if (pro && tile == 0) {
        Timed tm(c, kProfTransfer, st, pro_work);
        kb_prolong<T, true, false><<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B);
        pro = false;
    }
    while (nsweeps > 0) {
        const int ns = nsweeps >= 2 && (tile == 0 || tile_sweeps<T>() == 2) ? 2 : 1;
        // one colour (kb_gs): all of u and the faces, 1/D and b of that colour, its u written;
        // tiled: u, faces, 1/D and b once, u2 written once for ns sweeps (+ e of level t-1)
        const double b_in = ones ? 0.0 : 1.0;
        const Work w = tile == 0 ? work_of<T>(2.0 * ns * B * es * (Mc + 2.0 * Fc + (1.0 + 0.5 * b_in) * Mc),
                                              2.0 * ns * B * 5.0 * Mc)
                                 : work_of<T>(B * es * ((3.0 + b_in) * Mc + 2.0 * Fc + (pro ? 0.25 * Mc : 0.0)),
                                              B * (10.0 * ns * Mc + (pro ? 8.0 * Mc : 0.0)));
        Timed tm(c, kProfSmooth, st, w, tile == 0 ? 2 * ns : 1);
        if (tile == 0) {
            for (int h = 0; h < 2 * ns; ++h)
                kb_gs<T><<<grid_for(c, B * n * n / 2), 256, 0, st>>>(A, t, B, (first + h) & 1, ones);
            nsweeps -= ns;
            continue;
        }
        if constexpr (tile_sweeps<T>() == 2) {
            if (tile == 32) (ns == 2 ? launch_tile<T, 32, 2> : launch_tile<T, 32, 1>)(c, A, t, B, ones, first, pro, st);
            else if (tile == 16)
                (ns == 2 ? launch_tile<T, 16, 2> : launch_tile<T, 16, 1>)(c, A, t, B, ones, first, pro, st);
            else (ns == 2 ? launch_tile<T, 8, 2> : launch_tile<T, 8, 1>)(c, A, t, B, ones, first, pro, st);
        } else {
            if (tile == 32) launch_tile<T, 32, 1>(c, A, t, B, ones, first, pro, st);
            else if (tile == 16) launch_tile<T, 16, 1>(c, A, t, B, ones, first, pro, st);
            else launch_tile<T, 8, 1>(c, A, t, B, ones, first, pro, st);
        }
        swap_u(c, A, t);
        pro = false;
        nsweeps -= ns;
    }
    if (pro) {  // no sweeps at all: the correction alone
        Timed tm(c, kProfTransfer, st, pro_work);
        kb_prolong<T, true, false><<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B);
    }
}

// nsweeps sweeps of level t by the wavefront smoother, two per launch, u in
// place; post: the first launch adds P e first; pre: the last launch also
// writes the restricted residual into bc of level t-1.
mlqmc_status smooth_stream(mlqmc_ctx* c, const FmgArgs& A, int t, int B, int nsweeps, int first, int ones, bool pre,
                           bool post, cudaStream_t st)
{
    LevelTag lt(c, t);
    const int n = c->p.coarse_cells << t;
    const double Mc = cells_of(c, t), Fc = faces_of(c, t);
    while (nsweeps > 0) {
        const int ns = nsweeps >= 2 ? 2 : 1;
        const bool last = nsweeps == ns;
        const bool p = pre && last;
        Work w;
        w.bytes = 4.0 * B * ((ones ? 2.0 : 3.0) * Mc + 2.0 * Fc + (post ? 0.25 * Mc : 0.0) + (p ? 0.25 * Mc : 0.0));
        w.f32 = B * (10.0 * ns * Mc + (post ? 8.0 * Mc : 0.0) + (p ? 11.0 * Mc : 0.0));
        Timed tm(c, kProfSmooth, st, w);
        if (!mlqmc_stream::launch(A, t, n, B, ns, ones, first, p, post, st)) return MLQMC_ERR_CUDA;
        post = false;
        nsweeps -= ns;
    }
    return MLQMC_OK;
}

// nsweeps sweeps of level t by the TMA-fed tiled smoother, two per launch, u
// -> u2 swapped after each launch; pro: the first launch adds P e first.
// zin: u is zero on entry (first launch only reads no u).
// rr: the last launch also writes the restricted residual (bc of level t-1).
// Bytes per cell: u in, u2 out, b in (unless ones), kx and ky in, e in (pro, a
// quarter-size array) and the restricted residual out (rr, a quarter).
mlqmc_status smooth_tma(mlqmc_ctx* c, FmgArgs& A, int t, int B, int nsweeps, int first, int ones, bool pro,
                        cudaStream_t st, bool zin = false, bool rr = false)
{
    LevelTag lt(c, t);
    const int n = c->p.coarse_cells << t;
    const double Mc = cells_of(c, t), Fc = faces_of(c, t);
    while (nsweeps > 0) {
        const int ns = nsweeps >= 2 ? 2 : 1;
        const bool last_rr = rr && nsweeps == ns;
        const Work w = work_of<float>(
            4.0 * B * ((ones ? 2.0 : 3.0) * Mc - (zin ? Mc : 0.0) + 2.0 * Fc + (pro ? 0.25 * Mc : 0.0) +
                       (last_rr ? 0.25 * Mc : 0.0)),
            B * (10.0 * ns * Mc + (pro ? 8.0 * Mc : 0.0) + (last_rr ? 11.0 * Mc : 0.0)));
        Timed tm(c, kProfSmooth, st, w);
        if (!mlqmc_tma::launch(A, t, n, B, ns, ones, first, pro, zin, last_rr, c->sm_count, st))
            return MLQMC_ERR_CUDA;
        swap_u(c, A, t);
        pro = false;
        zin = false;
        nsweeps -= ns;
    }
    return MLQMC_OK;
}

// nsweeps sweeps of level t by the whole-sample smoother in one launch, u in
// place; pre: also the restricted residual; post: P e added first.
mlqmc_status smooth_whole(mlqmc_ctx* c, const FmgArgs& A, int t, int B, int nsweeps, int first, int ones, bool pre,
                          bool post, cudaStream_t st, bool zin = false)
{
    LevelTag lt(c, t);
    const int n = c->p.coarse_cells << t;
    const bool f64 = !is_mixed(c->p);
    const double Mc = cells_of(c, t), Fc = faces_of(c, t), es = f64 ? 8.0 : 4.0;
    Work w;
    w.bytes = es * B * ((ones ? 2.0 : 3.0) * Mc - (zin ? Mc : 0.0) + (f64 ? Mc : 0.0) + 2.0 * Fc +
                        (post ? 0.25 * Mc : 0.0) + (pre ? 0.25 * Mc : 0.0));
    const double fl = B * (10.0 * nsweeps * Mc + (post ? 8.0 * Mc : 0.0) + (pre ? 11.0 * Mc : 0.0));
    if (f64) w.f64 = fl;
    else w.f32 = fl;
    Timed tm(c, kProfSmooth, st, w);
    return mlqmc_whole::launch(A, t, n, B, nsweeps, ones, first, pre, post, zin, f64, st) ? MLQMC_OK : MLQMC_ERR_CUDA;
}

// Whether the pre-smoother of level t starts a correction from zero without
// reading u (so the V-cycle need not clear u first).
template <typename T>
bool zero_in_smoother(const mlqmc_ctx* c, int t, int B)
{
    const int sk = smoother_for(c, t, B);
    return c->p.nu1 > 0 && (sk == MLQMC_SMOOTHER_WHOLE || sk == MLQMC_SMOOTHER_TMA);
}

// Pre-smoothing of level t and the restricted residual into bc of level t-1.
// zin: u is zero on entry (a correction level below the cycle's top) and the
// smoother clears it itself (zero_in_smoother).
template <typename T>
mlqmc_status presmooth_restrict(mlqmc_ctx* c, FmgArgs& A, int t, int B, int top_ones, cudaStream_t st,
                                bool zin = false)
{
    LevelTag lt(c, t);
    const int sk = smoother_for(c, t, B);
    if (sk == MLQMC_SMOOTHER_WHOLE && c->p.nu1 > 0)  // residual and restriction in the same pass
        return smooth_whole(c, A, t, B, c->p.nu1, 0, top_ones, true, false, st, zin);
    if (sk == MLQMC_SMOOTHER_STREAM && c->p.nu1 > 0)  // residual and restriction fused into the last pass
        return smooth_stream(c, A, t, B, c->p.nu1, 0, top_ones, true, false, st);
    if (sk == MLQMC_SMOOTHER_TMA && c->p.nu1 > 0)  // the restricted residual fused into the last launch
        return smooth_tma(c, A, t, B, c->p.nu1, 0, top_ones, false, st, zin, true) == MLQMC_OK ? MLQMC_OK
                                                                                                : MLQMC_ERR_CUDA;
    smooth<T>(c, A, t, B, c->p.nu1, 0, top_ones, false, st);
    const int64_t n = c->p.coarse_cells << t;
    const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
    Timed tm(c, kProfTransfer, st, work_of<T>(B * es * ((top_ones ? 1.25 : 2.25) * Mc + 2.0 * Fc), B * 11.0 * Mc));
    kb_resid_restrict<T><<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B, top_ones);
    return last_error();
}

// Coarse-grid correction of level t and its post-smoothing.
template <typename T>
mlqmc_status correct_postsmooth(mlqmc_ctx* c, FmgArgs& A, int t, int B, int top_ones, cudaStream_t st)
{
    LevelTag lt(c, t);
    const int sk = smoother_for(c, t, B);
    if (sk == MLQMC_SMOOTHER_WHOLE && c->p.nu2 > 0)  // the correction in the same pass
        return smooth_whole(c, A, t, B, c->p.nu2, 1, top_ones, false, true, st);
    if (sk == MLQMC_SMOOTHER_STREAM && c->p.nu2 > 0)  // the correction fused into the first pass
        return smooth_stream(c, A, t, B, c->p.nu2, 1, top_ones, false, true, st);
    if (sk == MLQMC_SMOOTHER_TMA && c->p.nu2 > 0) return smooth_tma(c, A, t, B, c->p.nu2, 1, top_ones, true, st);
    smooth<T>(c, A, t, B, c->p.nu2, 1, top_ones, true, st);
    return last_error();
}

template <typename T>
mlqmc_status vcycle_batched(mlqmc_ctx* c, FmgArgs& A, int t_top, int B, bool ones, cudaStream_t st,
                            bool top_zero = false)
{
    for (int t = t_top; t >= 1; --t) {
        const int top_ones = (t == t_top && ones) ? 1 : 0;
        // a correction level (and, top_zero, the top level: the first cycle of a
        // refinement step) starts from zero: cleared here, or by its smoother
        const bool zero_entry = t < t_top || top_zero;
        const bool zin = zero_entry && zero_in_smoother<T>(c, t, B);
        if (zero_entry && !zin && zero_u(c, t, B, st) != MLQMC_OK) return MLQMC_ERR_CUDA;
        if (presmooth_restrict<T>(c, A, t, B, top_ones, st, zin) != MLQMC_OK) return MLQMC_ERR_CUDA;
    }
    {
        const double N0 = cells_of(c, 0), n0 = c->p.coarse_cells, es = sizeof(T);
        Timed tm(c, kProfSmallV, st, work_of<T>(B * es * (N0 * (n0 + 1.0) + 2.0 * N0), B * 4.0 * N0 * n0));
        LevelTag lt(c, 0);
        launch_coarse<T>(c, A, B, st);
    }
    for (int t = 1; t <= t_top; ++t) {
        const int top_ones = (t == t_top && ones) ? 1 : 0;
        if (correct_postsmooth<T>(c, A, t, B, top_ones, st) != MLQMC_OK) return MLQMC_ERR_CUDA;
    }
    return last_error();
}

// Residual norms, flags and the loop decision of one refinement pass on level t.
template <typename T>
mlqmc_status norms_and_ctl(mlqmc_ctx* c, const FmgArgs& A, int t, int B, int P, cudaGraphConditionalHandle h,
                           cudaStream_t st)
{
    const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
    {
        Timed tm(c, kProfReduce, st, work_of<double>(B * (8.0 * Mc + es * (2.0 * Fc + Mc) + 8.0), B * 12.0 * Mc));
        const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(B) * P, c->sm_count * 8));
        kb_resnorm_part<T><<<grid, 256, 0, st>>>(A, t, B, P, c->d_part);
    }
    {
        const int64_t n = c->p.coarse_cells << t;
        Timed tm(c, kProfReduce, st, work_of<double>(B * (8.0 * P + 12.0), B * 1.0 * P), 2);
        kb_norm_flags<<<grid_for(c, B), 256, 0, st>>>(c->d_part, P, c->d_norms, c->d_active, B,
                                                      c->p.refine_rtol * n, c->d_count);
        k_loop_ctl<<<1, 1, 0, st>>>(h, c->d_count, c->d_iters + t, c->p.refine_max_iter, c->d_status);
    }
    return last_error();
}

// The converged form's loop on level t inside a round capture: the first
// residual norms and the loop decision on the capture stream, then a
// conditional WHILE node whose body (captured on the body stream) runs the
// masked mu0 V-cycles, u64 += e, the next norms and the next decision. Same
// kernels and order as the host loop, without a host round trip per pass.
template <typename T>
mlqmc_status converge_device(mlqmc_ctx* c, FmgArgs& A, int t, int B, int P, cudaStream_t st)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    const int64_t n = c->p.coarse_cells << t;
    const double es = sizeof(T), Mc = cells_of(c, t);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    if (!ok(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &edges, &nd)) ||
        cs != cudaStreamCaptureStatusActive)
        return MLQMC_ERR_CUDA;
    cudaGraphConditionalHandle h{};
    if (!ok(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault))) return MLQMC_ERR_CUDA;
    if (!ok(cudaMemsetAsync(c->d_count, 0, sizeof(int), st)) ||
        !ok(cudaMemsetAsync(c->d_iters + t, 0, sizeof(int), st)))
        return MLQMC_ERR_CUDA;
    mlqmc_status s = norms_and_ctl<T>(c, A, t, B, P, h, st);
    if (s != MLQMC_OK) return s;
    if (!ok(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &edges, &nd))) return MLQMC_ERR_CUDA;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (!ok(cudaGraphAddNode(&node, cg, deps, edges, nd, &np))) return MLQMC_ERR_CUDA;
    cudaStream_t bs = G.body;
    if (!ok(cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal)))
        return MLQMC_ERR_CUDA;
    G.in_body = true;
    A.active = c->d_active;
    for (int m = 0; m < c->p.mu0 && s == MLQMC_OK; ++m) s = vcycle_batched<T>(c, A, t, B, false, bs, m == 0);
    if (s == MLQMC_OK) {
        Timed tm(c, kProfTransfer, bs, work_of<double>(B * (16.0 + es) * Mc, B * Mc));
        kb_update64<T><<<grid_for(c, B * n * n), 256, 0, bs>>>(A, t, B);
    }
    A.active = nullptr;
    if (s == MLQMC_OK) s = norms_and_ctl<T>(c, A, t, B, P, h, bs);
    G.in_body = false;
    cudaGraph_t body_out = nullptr;
    const bool ended = ok(cudaStreamEndCapture(bs, &body_out));
    if (s != MLQMC_OK) return s;
    if (!ended || !ok(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)))
        return MLQMC_ERR_CUDA;
    return MLQMC_OK;
}

// Host loop of the converged form on level t (refinement path): per-sample
// FP64 residual norms (r left in bc), active flags, then mu0 V-cycles on the
// correction of the active samples and u64 += e, until none is active.
template <typename T>
mlqmc_status converge_batched(mlqmc_ctx* c, FmgArgs& A, int t, int B, cudaStream_t st)
{
    LevelTag lt(c, t);
    const int64_t n = c->p.coarse_cells << t;
    const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
    // chunks of about 8192 cells per CTA (this path is never graph-captured: the buffer may grow here)
    const int P = static_cast<int>(std::max<int64_t>(1, n * n / 8192));
    if (static_cast<int64_t>(B) * P > c->part_cap) {
        cudaFree(c->d_part);
        c->d_part = nullptr;
        c->part_cap = 0;
        if (!ok(cudaMalloc(&c->d_part, sizeof(double) * static_cast<size_t>(B) * P))) return MLQMC_ERR_OOM;
        c->part_cap = static_cast<int64_t>(B) * P;
    }
    if (c->graph.round_capture) return converge_device<T>(c, A, t, B, P, st);
    for (int it = 0;; ++it) {
        {
            Timed tm(c, kProfReduce, st, work_of<double>(B * (8.0 * Mc + es * (2.0 * Fc + Mc) + 8.0), B * 12.0 * Mc));
            const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(B) * P, c->sm_count * 8));
            kb_resnorm_part<T><<<grid, 256, 0, st>>>(A, t, B, P, c->d_part);
        }
        if (!ok(cudaMemsetAsync(c->d_count, 0, sizeof(int), st))) return MLQMC_ERR_CUDA;
        {
            Timed tm(c, kProfReduce, st, work_of<double>(B * (8.0 * P + 12.0), B * 1.0 * P));
            kb_norm_flags<<<grid_for(c, B), 256, 0, st>>>(c->d_part, P, c->d_norms, c->d_active, B,
                                                          c->p.refine_rtol * n, c->d_count);
        }
        if (!ok(cudaMemcpyAsync(c->h_count, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaStreamSynchronize(st)))
            return MLQMC_ERR_CUDA;
        c->last_iters[t] = std::max(c->last_iters[t], it);
        if (*c->h_count == 0) break;
        if (it >= c->p.refine_max_iter) {
            c->host_status |= kStatusNotConverged;
            break;
        }
        A.active = c->d_active;
        mlqmc_status s = MLQMC_OK;
        for (int m = 0; m < c->p.mu0 && s == MLQMC_OK; ++m) s = vcycle_batched<T>(c, A, t, B, false, st, m == 0);
        if (s == MLQMC_OK) {
            Timed tm(c, kProfTransfer, st, work_of<double>(B * (16.0 + es) * Mc, B * Mc));
            kb_update64<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
        }
        A.active = nullptr;
        if (s != MLQMC_OK) return s;
    }
    return last_error();
}

// FMG stages 1..Lmax for the B_t samples that reach each level. Refinement
// path (mixed forms, converged FP64 form): solutions in u64, each stage starts
// with one correction step of mu0 V-cycles, then (rtol > 0) repeats it until
// converged. Otherwise (fixed-cycle FP64 form) mu0 V-cycles act on u itself.
template <typename T, bool MX>
mlqmc_status fmg_stages(mlqmc_ctx* c, FmgArgs& A, const int* Bt, int Lmax, double* d_usol, cudaStream_t st)
{
    const bool refine = A.refine != 0;
    // mixed forms with one refinement step per level: the step's u64 += e runs
    // inside the QoI kernel, which reads u64 anyway
    const bool fuse_update = MX && refine && !(c->p.refine_rtol > 0.0);
    size_t uoff = static_cast<size_t>(A.lv[0].n) * A.lv[0].n;
    // u64 written back by the fused update only when read later (centre QoI,
    // solution output); otherwise, on the TMA interpolation levels, the
    // interpolant itself travels in FP32 (interp32: in the level's field array)
    const int keep64 = (d_usol != nullptr || c->p.qoi != MLQMC_QOI_MEAN) ? 1 : 0;
    for (int t = 1; t <= Lmax; ++t) {
        const int B = Bt[t];
        if (B == 0) break;
        LevelTag lt(c, t);
        const int64_t n = c->p.coarse_cells << t;
        const double es = sizeof(T), Mc = cells_of(c, t), Fc = faces_of(c, t);
        const int interp32 = (fuse_update && !keep64 && mlqmc_resid::supported(static_cast<int>(n))) ? 1 : 0;
        if (refine && MX) {
            // the residual's 10 operations per cell run in FP32 error-free pairs: FP32 work
            Timed tm(c, kProfTransfer, st,
                     work_of<float>(B * (es * 0.25 * Mc + (interp32 ? 4.0 : 8.0) * Mc + es * (2.0 * Fc + Mc)),
                                    B * 10.0 * Mc));
            if (mlqmc_resid::supported(n)) {
                if (!mlqmc_resid::launch(A, t, n, B, interp32 != 0, c->sm_count, st)) return MLQMC_ERR_CUDA;
            } else {
                kb_prolong_resid64<<<grid_for(c, B * (n / 2) * (n / 2)), 256, 0, st>>>(A, t, B);
            }
        } else if (refine) {
            {
                Timed tm(c, kProfTransfer, st, work_of<T>(B * (es * 0.25 + 8.0) * Mc, B * 8.0 * Mc));
                kb_prolong<T, false, true><<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B);
            }
            {
                Timed tm(c, kProfTransfer, st, work_of<double>(B * (8.0 * Mc + es * (2.0 * Fc + Mc)), B * 10.0 * Mc));
                kb_resid64<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
            }
        }
        if (refine) {
            for (int m = 0; m < c->p.mu0; ++m) {
                mlqmc_status s = vcycle_batched<T>(c, A, t, B, false, st, m == 0);
                if (s != MLQMC_OK) return s;
            }
            if (!fuse_update) {
                Timed tm(c, kProfTransfer, st, work_of<double>(B * (16.0 + es) * Mc, B * Mc));
                kb_update64<T><<<grid_for(c, B * n * n), 256, 0, st>>>(A, t, B);
            }
            if (c->p.refine_rtol > 0.0) {
                mlqmc_status s = converge_batched<T>(c, A, t, B, st);
                if (s != MLQMC_OK) return s;
            }
        } else {
            {
                Timed tm(c, kProfTransfer, st, work_of<T>(B * es * 1.25 * Mc, B * 8.0 * Mc));
                kb_prolong<T, false, false><<<grid_for(c, B * n * n / 4), 256, 0, st>>>(A, t, B);
            }
            for (int m = 0; m < c->p.mu0; ++m) {
                mlqmc_status s = vcycle_batched<T>(c, A, t, B, true, st);
                if (s != MLQMC_OK) return s;
            }
        }
        {
            // bytes: u (or u64) read, the FP32 copy written; fused update: u64 also
            // written and the correction read (FP64: update and sum)
            const double qb = fuse_update ? (keep64 ? 24.0 : interp32 ? 12.0 : 16.0)
                                          : (refine ? 8.0 : es) + (refine && sizeof(T) == 4 ? 4.0 : 0.0);
            Timed tm(c, kProfReduce, st, work_of<double>(B * qb * Mc, B * (fuse_update ? 2.0 : 1.0) * Mc));
            if (n * n <= 4096) {  // one warp per sample
                const int grid = std::max(1, std::min((B + 7) / 8, c->sm_count * 16));
                if (fuse_update) kb_qoi<T, true, WarpTeam, MX><<<grid, 256, 0, st>>>(A, t, B, keep64);
                else if (refine) kb_qoi<T, true, WarpTeam><<<grid, 256, 0, st>>>(A, t, B, 1);
                else kb_qoi<T, false, WarpTeam><<<grid, 256, 0, st>>>(A, t, B, 1);
            } else {  // chunks of a sample over several CTAs, partial sums added in order
                const int P = qoi_chunks(c, t);
                const bool pass = fuse_update || (refine && sizeof(T) == 4) || c->p.qoi == MLQMC_QOI_MEAN;
                const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(B) * P, c->sm_count * 8));
                if (pass) {
                    if constexpr (MX) {
                        if (fuse_update) kb_qoi_part<T, true, true><<<grid, 256, 0, st>>>(A, t, B, P, c->d_qpart, keep64, interp32);
                        else kb_qoi_part<T, true, false><<<grid, 256, 0, st>>>(A, t, B, P, c->d_qpart, 1, 0);
                    } else {
                        if (refine) kb_qoi_part<T, true, false><<<grid, 256, 0, st>>>(A, t, B, P, c->d_qpart, 1, 0);
                        else kb_qoi_part<T, false, false><<<grid, 256, 0, st>>>(A, t, B, P, c->d_qpart, 1, 0);
                    }
                }
                if (refine) kb_qoi_final<T, true><<<grid_for(c, B), 256, 0, st>>>(A, t, B, P, c->d_qpart);
                else kb_qoi_final<T, false><<<grid_for(c, B), 256, 0, st>>>(A, t, B, P, c->d_qpart);
            }
        }
        if (d_usol) {
            Timed tm(c, kProfReduce, st, work_of<double>((8.0 + (refine ? 8.0 : es)) * Mc, 0.0));
            if (refine) kb_u_out<T, true><<<grid_for(c, n * n), 256, 0, st>>>(A, t, d_usol + uoff);
            else kb_u_out<T, false><<<grid_for(c, n * n), 256, 0, st>>>(A, t, d_usol + uoff);
            uoff += static_cast<size_t>(n) * n;
        }
    }
    return last_error();
}

// Default smoother per level: the FP32 wavefront where it fits, else the TMA
// tiles, else the plain tiles; FP64 form: the whole-sample smoother up to
// 64 x 64, kb_gs above (the FP64 plain tiles move less data but take longer:
// FP64 issue, not HBM, bounds these sweeps on GB300).
void default_smoothers(mlqmc_ctx* c)
{
    for (int t = 0; t < c->p.n_levels; ++t) {
        if (t == 0) c->smoother[t] = MLQMC_SMOOTHER_GS;
        else if (!is_mixed(c->p))  // FP64 form: a fixed rule, so every context gives the same bits
            c->smoother[t] = smoother_fits(c, MLQMC_SMOOTHER_WHOLE, t) ? MLQMC_SMOOTHER_WHOLE : MLQMC_SMOOTHER_GS;
        else if (smoother_fits(c, MLQMC_SMOOTHER_WHOLE, t)) c->smoother[t] = MLQMC_SMOOTHER_WHOLE;
        else if (smoother_fits(c, MLQMC_SMOOTHER_STREAM, t)) c->smoother[t] = MLQMC_SMOOTHER_STREAM;
        else if (smoother_fits(c, MLQMC_SMOOTHER_TMA, t)) c->smoother[t] = MLQMC_SMOOTHER_TMA;
        else c->smoother[t] = MLQMC_SMOOTHER_TILE;
        c->smoother_small[t] = c->smoother[t];
        c->kl_nt[t][0] = c->kl_nt[t][1] = mlqmc_kl::tile_samples();
    }
}

// Autotuner (mixed forms): for every level that more than one smoother can
// run, time one V-cycle visit of the level (pre-smoothing and the restricted
// residual, correction and post-smoothing) of each candidate on 1024 samples
// of zeroed scratch pools (the timing does not depend on the values) and keep
// the fastest. Runs once, at creation, on its own stream. The FP64 form takes
// a fixed rule instead (default_smoothers).
mlqmc_status tune_smoothers(mlqmc_ctx* c)
{
    default_smoothers(c);
    const bool f64 = !is_mixed(c->p);
    if (f64) return MLQMC_OK;
    const int64_t launches0 = c->launches;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) || !ok(cudaEventCreate(&e0)) ||
        !ok(cudaEventCreate(&e1)))
        return MLQMC_ERR_CUDA;
    mlqmc_status res = MLQMC_OK;
    const int all[4] = {MLQMC_SMOOTHER_GS, MLQMC_SMOOTHER_WHOLE, MLQMC_SMOOTHER_STREAM, MLQMC_SMOOTHER_TMA};
    int large_best[MLQMC_MAX_LEVELS] = {};
    for (int t = 1; t < c->p.n_levels && res == MLQMC_OK; ++t)
    for (int cls = 1; cls >= 0 && res == MLQMC_OK; --cls) {  // large batches, then small ones
        int cands[4], nc = 0;
        for (int k : all)
            if ((f64 || k != MLQMC_SMOOTHER_GS) && smoother_fits(c, k, t)) cands[nc++] = k;
        if (nc < 2) continue;
        int64_t B = cls ? 1024 : 64;  // the same for every context, whatever its max_samples
        const size_t per = level_bytes_per_sample(c->p, c->Ka, t) + level_bytes_per_sample(c->p, c->Ka, t - 1);
        while (B > 64 && per * static_cast<size_t>(B) > c->pool_budget / 4) B /= 2;
        if (ensure_pool(c, t - 1, B) != MLQMC_OK || ensure_pool(c, t, B) != MLQMC_OK) {
            res = MLQMC_ERR_OOM;
            break;
        }
        for (int u = t - 1; u <= t; ++u) {
            const LevelPool& P = c->pools[u];
            const size_t bytes = level_bytes_per_sample(c->p, c->Ka, u) * static_cast<size_t>(P.cap);
            if (!ok(cudaMemsetAsync(P.mem, 0, bytes, st))) res = MLQMC_ERR_CUDA;
        }
        double* tms = cls ? c->tune_ms[t] : c->tune_small_ms[t];
        int best = cands[0];
        for (int k = 0; k < nc && res == MLQMC_OK; ++k) {
            c->smoother[t] = c->smoother_small[t] = cands[k];
            FmgArgs A = base_args(c);
            float ms = 0.0f, tot = 0.0f;
            for (int rep = 0; rep < 4 && res == MLQMC_OK; ++rep) {  // one untimed visit, then three timed
                if (!ok(cudaEventRecord(e0, st))) res = MLQMC_ERR_CUDA;
                if (res == MLQMC_OK)
                    res = f64 ? presmooth_restrict<double>(c, A, t, static_cast<int>(B), 0, st)
                              : presmooth_restrict<float>(c, A, t, static_cast<int>(B), 0, st);
                if (res == MLQMC_OK)
                    res = f64 ? correct_postsmooth<double>(c, A, t, static_cast<int>(B), 0, st)
                              : correct_postsmooth<float>(c, A, t, static_cast<int>(B), 0, st);
                if (res == MLQMC_OK && (!ok(cudaEventRecord(e1, st)) || !ok(cudaEventSynchronize(e1)) ||
                                        !ok(cudaEventElapsedTime(&ms, e0, e1))))
                    res = MLQMC_ERR_CUDA;
                if (rep > 0) tot += ms;
            }
            tms[cands[k]] = tot / 3.0;
            if (tms[cands[k]] < tms[best]) best = cands[k];
        }
        if (cls) {
            large_best[t] = best;
        } else {
            c->smoother[t] = large_best[t];
            c->smoother_small[t] = best;
        }
    }
    if (res == MLQMC_OK && !ok(cudaStreamSynchronize(st))) res = MLQMC_ERR_CUDA;
    if (res == MLQMC_OK && c->host_status == 0) {
        int dev = 0;
        if (!ok(cudaMemcpy(&dev, c->d_status, sizeof(int), cudaMemcpyDeviceToHost))) res = MLQMC_ERR_CUDA;
        else if (dev != 0) res = MLQMC_ERR_DEVICE_STATUS;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    c->launches = launches0;
    if (res != MLQMC_OK) default_smoothers(c);
    return res;
}

// Autotuner of the tensor-core KL tile width (mixed forms): for every level
// with the contraction, time one launch with 128 and with 256 samples per
// tile on up to 262,144 of the level's cells (the per-tile work is the
// level's own) for 64 and for 256 samples (the small- and large-batch
// classes), zeroed C operand, scratch output; keep the faster width per class.
mlqmc_status tune_kl(mlqmc_ctx* c)
{
    if (!c->kl_tc) return MLQMC_OK;
    const int Bs[2] = {64, 256}, NTs[2] = {128, 256};
    int64_t maxM = 0;
    for (int t = 0; t < c->p.n_levels; ++t)
        if (c->d_psi_tc[t]) {
            const int64_t n = c->p.coarse_cells << t;
            maxM = std::max<int64_t>(maxM, std::min<int64_t>(n * n, 262144));
        }
    if (maxM == 0) return MLQMC_OK;
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mlqmc_status res = MLQMC_OK;
    if (!ok(cudaMalloc(&out, sizeof(float) * static_cast<size_t>(maxM) * Bs[1]))) {
        cudaGetLastError();
        return MLQMC_ERR_OOM;
    }
    if (!ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) || !ok(cudaEventCreate(&e0)) ||
        !ok(cudaEventCreate(&e1)) ||
        !ok(cudaMemsetAsync(c->d_C, 0, static_cast<size_t>(c->max_samples) *
                                           mlqmc_kl::row_bytes(c->kl_variant, c->p.n_modes), st)))
        res = MLQMC_ERR_CUDA;
    for (int t = 0; t < c->p.n_levels && res == MLQMC_OK; ++t) {
        if (!c->d_psi_tc[t]) continue;
        const int64_t n = c->p.coarse_cells << t;
        const int M = static_cast<int>(std::min<int64_t>(n * n, 262144));
        for (int cls = 0; cls < 2 && res == MLQMC_OK; ++cls) {
            for (int k = 0; k < 2 && res == MLQMC_OK; ++k) {
                float ms = 0.0f, tot = 0.0f;
                for (int rep = 0; rep < 4 && res == MLQMC_OK; ++rep) {  // one untimed launch, then three timed
                    if (!ok(cudaEventRecord(e0, st)) ||
                        !mlqmc_kl::launch(c->kl_variant, c->kl_maps[t], M, Bs[cls], c->p.n_modes, out,
                                          static_cast<size_t>(M), c->d_status, st, NTs[k]) ||
                        !ok(cudaEventRecord(e1, st)) || !ok(cudaEventSynchronize(e1)) ||
                        !ok(cudaEventElapsedTime(&ms, e0, e1)))
                        res = MLQMC_ERR_CUDA;
                    if (rep > 0) tot += ms;
                }
                c->tune_kl_ms[t][cls][k] = tot / 3.0;
            }
            c->kl_nt[t][cls] = c->tune_kl_ms[t][cls][0] < c->tune_kl_ms[t][cls][1] ? NTs[0] : NTs[1];
        }
    }
    if (res == MLQMC_OK && !ok(cudaStreamSynchronize(st))) res = MLQMC_ERR_CUDA;
    if (res == MLQMC_OK) {
        int dev = 0;
        if (!ok(cudaMemcpy(&dev, c->d_status, sizeof(int), cudaMemcpyDeviceToHost))) res = MLQMC_ERR_CUDA;
        else if (dev != 0) res = MLQMC_ERR_DEVICE_STATUS;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    if (res != MLQMC_OK)
        for (int t = 0; t < c->p.n_levels; ++t) c->kl_nt[t][0] = c->kl_nt[t][1] = mlqmc_kl::tile_samples();
    return res;
}

// Everything for one chunk of samples already staged in d_samples (rank order).
mlqmc_status run_chunk(mlqmc_ctx* c, int count, const int* Bt, int Lmax, double* d_sums, double* d_Fout,
                       double* d_usol, cudaStream_t st)
{
    const mlqmc_problem& p = c->p;
    for (int t = 0; t <= Lmax; ++t) {
        mlqmc_status s = ensure_pool(c, t, Bt[t]);
        if (s != MLQMC_OK) return s;
    }
    FmgArgs A = base_args(c);
    mlqmc_status s = MLQMC_OK;
    const int kpad = c->kl_tc ? static_cast<int>(mlqmc_kl::row_bytes(c->kl_variant, p.n_modes) / 4) : 0;
    // every level's field from the tensor cores: the normals and the FP32
    // coefficients of the SIMT synthesis are not read
    bool all_tc = true;
    for (int t = 0; t <= Lmax; ++t) all_tc = all_tc && uses_tc(c, t);
    if (is_mixed(p) && !c->matern && c->kl_tc && c->kl_variant == mlqmc_kl::Variant::TF32 &&
        static_cast<int64_t>(count) * kpad < (int64_t{1} << 31)) {
        // normals, FP32 coefficients and the C operand in one pass
        const int64_t total = static_cast<int64_t>(count) * kpad;
        Timed tm(c, kProfPoints, st,
                 work_of<float>(static_cast<double>(count) * (p.n_modes * (all_tc ? 0.0 : 12.0) + kpad * 4.0 +
                                                              sizeof(SampleDesc)),
                                0.0));
        k_points_mixed<<<grid_for(c, total), 256, 0, st>>>(
            c->d_samples, count, p.n_modes, kpad, FastDiv(static_cast<uint32_t>(kpad)), p.sampler, p.seed, c->d_z,
            c->d_shift, p.n_shifts, c->d_sqrt_theta, all_tc ? nullptr : c->d_Y, all_tc ? nullptr : c->d_c32,
            static_cast<float*>(c->d_C));
        if (last_error() != MLQMC_OK) return MLQMC_ERR_CUDA;
        c->c32_ready = !all_tc;
    } else {
        s = launch_points(c, c->d_samples, count, c->d_Y, nullptr, st);
        if (s != MLQMC_OK) return s;
        s = build_c(c, count, st);
        if (s != MLQMC_OK) return s;
    }
    // mixed forms, separable modes: FP32 coefficients of all the chunk's
    // samples once, before both streams' SIMT syntheses read them
    if (is_mixed(p) && !c->matern && !c->c32_ready && !all_tc) {
        Timed tm(c, kProfSynth, st, work_of<double>(count * 12.0 * p.n_modes, count * 1.0 * p.n_modes));
        k_coef32<<<grid_for(c, static_cast<int64_t>(count) * p.n_modes), 256, 0, st>>>(A, count, c->d_sqrt_theta,
                                                                                        c->d_c32);
        c->c32_ready = true;
    }
    // level 0 (field, faces, factorisation and exact solve: latency-bound,
    // one thread per sample) on the side stream while the main stream
    // synthesises levels 1..Lmax; joined before the FMG stages
    if (!ok(cudaEventRecord(c->ev_fork, st)) || !ok(cudaStreamWaitEvent(c->side, c->ev_fork, 0))) {
        c->c32_ready = false;
        return MLQMC_ERR_CUDA;
    }
    s = is_mixed(p) ? synth_batched<float>(c, A, 0, Bt[0], c->side) : synth_batched<double>(c, A, 0, Bt[0], c->side);
    if (is_mixed(p) && all_tc) {
        // the persistent contractions cannot start beside the factorisation's
        // CTAs (both need most of an SM's shared memory): the main stream
        // issues the other levels' contractions first, the factorisation
        // follows them and runs beside those levels' faces
        for (int t = 1; s == MLQMC_OK && t <= Lmax && Bt[t] > 0; ++t)
            s = synth_batched<float>(c, A, t, Bt[t], st, SynthPart::field);
        if (!ok(cudaEventRecord(c->ev_fields, st)) || !ok(cudaStreamWaitEvent(c->side, c->ev_fields, 0)))
            s = MLQMC_ERR_CUDA;
        if (s == MLQMC_OK) s = launch_level0(c, A, Bt[0], c->side);
        if (!ok(cudaEventRecord(c->ev_join, c->side))) s = MLQMC_ERR_CUDA;
        for (int t = 1; s == MLQMC_OK && t <= Lmax && Bt[t] > 0; ++t)
            s = synth_batched<float>(c, A, t, Bt[t], st, SynthPart::faces);
    } else {
        if (s == MLQMC_OK) s = launch_level0(c, A, Bt[0], c->side);
        if (!ok(cudaEventRecord(c->ev_join, c->side))) s = MLQMC_ERR_CUDA;
        for (int t = 1; s == MLQMC_OK && t <= Lmax && Bt[t] > 0; ++t)
            s = is_mixed(p) ? synth_batched<float>(c, A, t, Bt[t], st) : synth_batched<double>(c, A, t, Bt[t], st);
    }
    if (!ok(cudaStreamWaitEvent(st, c->ev_join, 0)) && s == MLQMC_OK) s = MLQMC_ERR_CUDA;
    c->c32_ready = false;
    if (s != MLQMC_OK) return s;
    if (d_usol) {
        const int64_t n0 = p.coarse_cells;
        Timed tm(c, kProfReduce, st, work_of<double>(16.0 * n0 * n0, 0.0));
        if (is_mixed(p)) kb_u_out<float, true><<<grid_for(c, n0 * n0), 256, 0, st>>>(A, 0, d_usol);
        else if (A.refine) kb_u_out<double, true><<<grid_for(c, n0 * n0), 256, 0, st>>>(A, 0, d_usol);
        else kb_u_out<double, false><<<grid_for(c, n0 * n0), 256, 0, st>>>(A, 0, d_usol);
    }
    s = is_mixed(p) ? fmg_stages<float, true>(c, A, Bt, Lmax, d_usol, st)
                    : fmg_stages<double, false>(c, A, Bt, Lmax, d_usol, st);
    if (s != MLQMC_OK) return s;
    if (d_sums) {
        Timed tm(c, kProfReduce, st, work_of<double>(count * (8.0 * p.n_levels + sizeof(SampleDesc)), count * 2.0 * p.n_levels));
        k_sums<<<p.n_levels * p.n_shifts, 256, 0, st>>>(c->d_samples, count, c->d_F, p.n_levels, p.n_shifts, p.reuse,
                                                        d_sums);
    }
    if (d_Fout) {
        Timed tm(c, kProfReduce, st, work_of<double>(count * (16.0 * p.n_levels + sizeof(SampleDesc)), 0.0));
        k_fout<<<grid_for(c, static_cast<int64_t>(count) * p.n_levels), 256, 0, st>>>(c->d_samples, count, c->d_F,
                                                                                      p.n_levels, d_Fout);
    }
    return last_error();
}

// Upload `count` descriptors (rank order) from host memory.
mlqmc_status stage_samples(mlqmc_ctx* c, const SampleDesc* src, int count, cudaStream_t st)
{
    if (!ok(cudaEventSynchronize(c->staged))) return MLQMC_ERR_CUDA;
    std::memcpy(c->h_samples, src, static_cast<size_t>(count) * sizeof(SampleDesc));
    if (count > 0 &&
        (!ok(cudaMemcpyAsync(c->d_samples, c->h_samples, count * sizeof(SampleDesc), cudaMemcpyHostToDevice, st)) ||
         !ok(cudaEventRecord(c->staged, st))))
        return MLQMC_ERR_CUDA;
    return MLQMC_OK;
}

void free_ctx(mlqmc_ctx* c)
{
    if (!c) return;
    cudaFree(c->d_psi);
    cudaFree(c->d_psi32);
    cudaFree(c->d_mix_F);
    cudaFree(c->d_mix_S);
    cudaFree(c->d_mix_W);
    cudaFree(c->d_grp_start);
    cudaFree(c->d_grp_b);
    cudaFree(c->d_grp_m);
    cudaFree(c->d_grp_sqrt);
    cudaFree(c->d_z);
    cudaFree(c->d_shift);
    cudaFree(c->d_ma);
    cudaFree(c->d_mb);
    cudaFree(c->d_sqrt_theta);
    for (auto* q : c->d_psi_tc) cudaFree(q);
    cudaFree(c->d_C);
    cudaFree(c->d_samples);
    cudaFree(c->d_Y);
    cudaFree(c->d_F);
    cudaFree(c->d_chol);
    cudaFree(c->d_chol32);
    cudaFree(c->d_norms);
    cudaFree(c->d_active);
    cudaFree(c->d_count);
    cudaFree(c->d_status);
    cudaFree(c->d_queue);
    cudaFree(c->d_iters);
    for (auto& P : c->pools) cudaFree(P.mem);
    if (c->staged) cudaEventDestroy(c->staged);
    cudaFree(c->d_psi_dense);
    cudaFree(c->d_part);
    cudaFree(c->d_qpart);
    cudaFree(c->d_c32);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_fields) cudaEventDestroy(c->ev_fields);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto& m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->h_samples) cudaFreeHost(c->h_samples);
    if (c->h_count) cudaFreeHost(c->h_count);
    if (c->h_status) cudaFreeHost(c->h_status);
    delete c;
}

template <typename X>
bool dev_upload(X** dst, const X* src, size_t cnt)
{
    if (!ok(cudaMalloc(dst, std::max<size_t>(1, cnt) * sizeof(X)))) return false;
    return cnt == 0 || ok(cudaMemcpy(*dst, src, cnt * sizeof(X), cudaMemcpyHostToDevice));
}

mlqmc_status check_problem(const mlqmc_problem* p)
{
    if (!p) return MLQMC_ERR_INVALID_ARG;
    if (p->n_levels < 1 || p->n_levels > MLQMC_MAX_LEVELS) return MLQMC_ERR_INVALID_ARG;
    if (p->coarse_cells < 2 || (p->coarse_cells & 1) || p->coarse_cells > 16) return MLQMC_ERR_INVALID_ARG;
    if (static_cast<int64_t>(p->coarse_cells) << (p->n_levels - 1) > 4096) return MLQMC_ERR_INVALID_ARG;
    if (p->n_modes < 1 || p->n_modes > MLQMC_MAX_MODES) return MLQMC_ERR_INVALID_ARG;
    if (!(p->sigma > 0.0) || !(p->corr_len > 0.0)) return MLQMC_ERR_INVALID_ARG;
    if (p->qoi != MLQMC_QOI_CENTER && p->qoi != MLQMC_QOI_MEAN) return MLQMC_ERR_INVALID_ARG;
    if (p->mu0 < 1 || p->nu1 < 0 || p->nu2 < 0 || p->mu0 > 64 || p->nu1 > 64 || p->nu2 > 64) return MLQMC_ERR_INVALID_ARG;
    if (p->precision < MLQMC_FP64 || p->precision > MLQMC_MIXED_BF16X3) return MLQMC_ERR_INVALID_ARG;
    if (p->refine_rtol < 0.0 || p->refine_max_iter < 0) return MLQMC_ERR_INVALID_ARG;
    if (p->sampler != MLQMC_SAMPLER_MC && p->sampler != MLQMC_SAMPLER_LATTICE) return MLQMC_ERR_INVALID_ARG;
    if (p->n_shifts < 1 || p->n_shifts > 4096) return MLQMC_ERR_INVALID_ARG;
    if (p->reuse != 0 && p->reuse != 1) return MLQMC_ERR_INVALID_ARG;
    if (p->covariance != MLQMC_COV_SEPARABLE_EXP && p->covariance != MLQMC_COV_MATERN) return MLQMC_ERR_INVALID_ARG;
    if (p->covariance == MLQMC_COV_MATERN) {
        if (!mlqmc_matern::supported_nu(p->matern_nu) || p->nystrom_m < 2 || p->nystrom_m > 128 ||
            !p->nystrom_theta || !p->nystrom_psi || p->n_modes > p->nystrom_m * p->nystrom_m)
            return MLQMC_ERR_INVALID_ARG;
        for (int j = 0; j < p->n_modes; ++j)
            if (!(p->nystrom_theta[j] > 0.0)) return MLQMC_ERR_INVALID_ARG;
    }
    if (p->sampler == MLQMC_SAMPLER_LATTICE) {
        if (!p->genvec || p->log2_nmax < 0 || p->log2_nmax > 32) return MLQMC_ERR_INVALID_ARG;
        for (int j = 0; j < p->n_modes; ++j)
            if ((p->genvec[j] & 1u) == 0) return MLQMC_ERR_INVALID_ARG;
    }
    return MLQMC_OK;
}

// Separable exponential covariance: the s largest products of the closed-form
// 1D eigenpairs (Sec. 5), each level's 1D tables and the modes grouped by
// their first index for the separable synthesis.
mlqmc_status setup_separable(mlqmc_ctx* c, const mlqmc_problem* p)
{
    c->modes = mlqmc::select_modes(p->corr_len, p->sigma, p->n_modes);
    const int K1 = c->modes.K1;
    c->eig = mlqmc::kl_eigen_1d(p->corr_len, K1);
    int Ka = 0;
    for (int m = 0; m < p->n_modes; ++m) Ka = std::max(Ka, c->modes.a[m] + 1);
    c->Ka = Ka;
    std::vector<int> gstart(Ka + 1, 0), gb, gm;
    std::vector<double> gsq;
    for (int a = 0; a < Ka; ++a) {
        gstart[a] = static_cast<int>(gb.size());
        for (int m = 0; m < p->n_modes; ++m)
            if (c->modes.a[m] == a) {
                gb.push_back(c->modes.b[m]);
                gm.push_back(m);
                gsq.push_back(std::sqrt(c->modes.theta[m]));
            }
    }
    gstart[Ka] = static_cast<int>(gb.size());
    std::vector<double> psi_all, tab;
    size_t off = 0;
    for (int t = 0; t < p->n_levels; ++t) {
        const int n = p->coarse_cells << t;
        mlqmc::psi_table(c->eig, p->corr_len, K1, n, tab);
        c->psi_off[t] = off;
        psi_all.insert(psi_all.end(), tab.begin(), tab.end());
        off += tab.size();
    }
    std::vector<float> psi32(psi_all.begin(), psi_all.end());
    std::vector<double> sq(p->n_modes);
    for (int m = 0; m < p->n_modes; ++m) sq[m] = std::sqrt(c->modes.theta[m]);
    bool good = dev_upload(&c->d_psi, psi_all.data(), psi_all.size()) &&
                dev_upload(&c->d_psi32, psi32.data(), psi32.size()) &&
                dev_upload(&c->d_grp_start, gstart.data(), gstart.size()) &&
                dev_upload(&c->d_grp_b, gb.data(), gb.size()) && dev_upload(&c->d_grp_m, gm.data(), gm.size()) &&
                dev_upload(&c->d_grp_sqrt, gsq.data(), gsq.size()) &&
                dev_upload(&c->d_z, c->z.data(), c->z.size()) &&
                dev_upload(&c->d_ma, c->modes.a.data(), c->modes.a.size()) &&
                dev_upload(&c->d_mb, c->modes.b.data(), c->modes.b.size()) &&
                dev_upload(&c->d_sqrt_theta, sq.data(), sq.size());
    return good ? MLQMC_OK : MLQMC_ERR_OOM;
}

// Matern covariance: the caller's Nystrom eigenpairs at the nodes, every
// level's modes at its cell centres by the Nystrom interpolation formula
// (Sec. 5), FP64 on the device, once.
mlqmc_status setup_matern(mlqmc_ctx* c, const mlqmc_problem* p)
{
    const int s = p->n_modes, m = p->nystrom_m, M = m * m;
    c->modes.theta.assign(p->nystrom_theta, p->nystrom_theta + s);
    c->modes.a.assign(s, -1);
    c->modes.b.assign(s, -1);
    c->modes.K1 = 0;
    c->Ka = 1;
    // FNV-1a of the nodal eigenfunctions: contexts of one multi-index run must share them
    uint64_t h = 1469598103934665603ull;
    const unsigned char* bytes = reinterpret_cast<const unsigned char*>(p->nystrom_psi);
    for (size_t i = 0; i < static_cast<size_t>(M) * s * sizeof(double); ++i) h = (h ^ bytes[i]) * 1099511628211ull;
    c->psi_hash = h;
    std::vector<double> wpsi(static_cast<size_t>(M) * s), sq(s);
    for (int q = 0; q < M; ++q)
        for (int j = 0; j < s; ++j)
            wpsi[static_cast<size_t>(q) * s + j] = p->nystrom_psi[static_cast<size_t>(q) * s + j] / M / p->nystrom_theta[j];
    for (int j = 0; j < s; ++j) sq[j] = std::sqrt(p->nystrom_theta[j]);
    size_t total = 0;
    for (int t = 0; t < p->n_levels; ++t) {
        const size_t n = static_cast<size_t>(p->coarse_cells) << t;
        c->dense_off[t] = total;
        total += n * n * s;
    }
    const std::vector<int> zeros(s, 0), gstart(2, 0);
    const double one = 0.0;
    const float one32 = 0.0f;
    double* d_wpsi = nullptr;
    bool good = dev_upload(&d_wpsi, wpsi.data(), wpsi.size()) && ok(cudaMalloc(&c->d_psi_dense, total * sizeof(double))) &&
                dev_upload(&c->d_psi, &one, 1) && dev_upload(&c->d_psi32, &one32, 1) &&
                dev_upload(&c->d_grp_start, gstart.data(), gstart.size()) &&
                dev_upload(&c->d_z, c->z.data(), c->z.size()) && dev_upload(&c->d_ma, zeros.data(), zeros.size()) &&
                dev_upload(&c->d_mb, zeros.data(), zeros.size()) && dev_upload(&c->d_sqrt_theta, sq.data(), sq.size());
    if (!good) {
        cudaFree(d_wpsi);
        return MLQMC_ERR_OOM;
    }
    for (int t = 0; good && t < p->n_levels; ++t)
        good = mlqmc_matern::interpolate(p->matern_nu, p->corr_len, p->sigma, m, s, d_wpsi,
                                         p->coarse_cells << t, c->d_psi_dense + c->dense_off[t], 0);
    good = good && ok(cudaDeviceSynchronize());
    cudaFree(d_wpsi);
    return good ? MLQMC_OK : MLQMC_ERR_CUDA;
}

// Samples per level count of a rank-ordered range: B[t] = #{level >= t}.
void count_levels(const SampleDesc* s, int count, int n_levels, int* Bt, int* Lmax)
{
    for (int t = 0; t < n_levels; ++t) Bt[t] = 0;
    *Lmax = -1;
    for (int q = 0; q < count; ++q) {
        for (int t = 0; t <= s[q].level; ++t) Bt[t]++;
        *Lmax = std::max(*Lmax, s[q].level);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" mlqmc_status mlqmc_create(const mlqmc_problem* p, int64_t max_samples_per_call, mlqmc_ctx** out)
{
    if (!out) return MLQMC_ERR_INVALID_ARG;
    *out = nullptr;
    mlqmc_status st = check_problem(p);
    if (st != MLQMC_OK) return st;
    if (max_samples_per_call < 0) return MLQMC_ERR_INVALID_ARG;
    mlqmc_ctx* c = new (std::nothrow) mlqmc_ctx();
    if (!c) return MLQMC_ERR_OOM;
    c->p = *p;
    if (!ok(cudaGetDevice(&c->device)) ||
        !ok(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device))) {
        free_ctx(c);
        return MLQMC_ERR_CUDA;
    }
    if (p->sampler == MLQMC_SAMPLER_LATTICE) c->z.assign(p->genvec, p->genvec + p->n_modes);
    else c->z.assign(p->n_modes, 1u);
    c->p.genvec = nullptr;

    // KL tables (Sec. 5)
    c->matern = p->covariance == MLQMC_COV_MATERN;
    c->p.nystrom_theta = nullptr;
    c->p.nystrom_psi = nullptr;
    mlqmc_status kst = c->matern ? setup_matern(c, p) : setup_separable(c, p);
    if (kst != MLQMC_OK) {
        free_ctx(c);
        return kst;
    }
    // lattice shift table, while it stays small (up to 2^22 entries, 32 MB)
    if (p->sampler == MLQMC_SAMPLER_LATTICE &&
        static_cast<int64_t>(p->n_shifts) * p->n_levels * p->n_modes <= (int64_t{1} << 22)) {
        const int64_t total = static_cast<int64_t>(p->n_shifts) * p->n_levels * p->n_modes;
        if (!ok(cudaMalloc(&c->d_shift, static_cast<size_t>(total) * sizeof(uint64_t)))) {
            free_ctx(c);
            return MLQMC_ERR_OOM;
        }
        k_shift_table<<<static_cast<int>(std::min<int64_t>((total + 255) / 256, 4096)), 256>>>(
            p->n_shifts, p->n_levels, p->n_modes, p->seed, c->d_shift);
        if (!ok(cudaGetLastError()) || !ok(cudaDeviceSynchronize())) {
            free_ctx(c);
            return MLQMC_ERR_CUDA;
        }
    }

    // per-chunk buffers
    c->max_samples = max_samples_per_call > 0 ? max_samples_per_call : 65536;
    const size_t ms = static_cast<size_t>(c->max_samples);
    const size_t N0 = static_cast<size_t>(p->coarse_cells) * p->coarse_cells;
    c->chol_stride = align256(sizeof(double) * N0 * (p->coarse_cells + 1));
    bool good = ok(cudaMalloc(&c->d_samples, ms * sizeof(SampleDesc))) &&
           ok(cudaMalloc(&c->d_Y, ms * p->n_modes * sizeof(double))) &&
           (p->precision == MLQMC_FP64 || ok(cudaMalloc(&c->d_c32, ms * p->n_modes * sizeof(float)))) &&
           ok(cudaMalloc(&c->d_F, ms * p->n_levels * sizeof(double))) &&
           ok(cudaMalloc(&c->d_chol, ms * c->chol_stride)) && ok(cudaMalloc(&c->d_chol32, ms * c->chol_stride / 2)) &&
           ok(cudaMalloc(&c->d_norms, ms * sizeof(double))) &&
           ok(cudaMalloc(&c->d_active, ms * sizeof(int))) && ok(cudaMalloc(&c->d_count, sizeof(int))) &&
           ok(cudaMallocHost(&c->h_samples, ms * sizeof(SampleDesc))) &&
           ok(cudaMallocHost(&c->h_count, sizeof(int))) && ok(cudaMallocHost(&c->h_status, sizeof(int))) &&
           ok(cudaMalloc(&c->d_status, sizeof(int))) &&
           ok(cudaMalloc(&c->d_queue, sizeof(int))) && ok(cudaMemset(c->d_status, 0, sizeof(int))) &&
           ok(cudaMalloc(&c->d_iters, 2 * MLQMC_MAX_LEVELS * sizeof(int))) &&
           ok(cudaMemset(c->d_iters, 0, 2 * MLQMC_MAX_LEVELS * sizeof(int))) &&
           ok(cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming)) &&
           ok(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) &&
           ok(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&c->ev_fields, cudaEventDisableTiming));
    if (!good) {
        free_ctx(c);
        return MLQMC_ERR_OOM;
    }

    // shared memory of the tiled smoother
    if (!(tile_attrs<32>() && tile_attrs<16>() && tile_attrs<8>() && mlqmc_stream::prepare() &&
          ok(cudaFuncSetAttribute(kb_level0_fixed<float, true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(level0_smem<8>()))) &&
          ok(cudaFuncSetAttribute(kb_level0_fixed<double, false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(level0_smem<8>()))))) {
        free_ctx(c);
        return MLQMC_ERR_CUDA;
    }
    // tensor-core KL tables (mixed forms): Psi of every level, its rows padded
    // with zeros to whole 128-cell tiles (the contraction stores only the
    // level's cells)
    if (p->precision == MLQMC_MIXED_TF32 || p->precision == MLQMC_MIXED_BF16X3) {
        c->kl_variant = p->precision == MLQMC_MIXED_TF32 ? mlqmc_kl::Variant::TF32 : mlqmc_kl::Variant::BF16X3;
        const size_t rb = mlqmc_kl::row_bytes(c->kl_variant, p->n_modes);
        good = mlqmc_kl::prepare_kernel() && ok(cudaMalloc(&c->d_C, ms * rb));
        for (int t = 0; good && t < p->n_levels; ++t) {
            const int n = p->coarse_cells << t;
            const int mpad = (n * n + 127) / 128 * 128;
            good = ok(cudaMalloc(&c->d_psi_tc[t], static_cast<size_t>(mpad) * rb)) &&
                   ok(cudaMemset(c->d_psi_tc[t], 0, static_cast<size_t>(mpad) * rb)) &&
                   (c->matern ? mlqmc_kl::build_psi_dense(c->kl_variant, c->d_psi_dense + c->dense_off[t],
                                                          static_cast<int64_t>(n) * n, p->n_modes, c->d_psi_tc[t], 0)
                              : mlqmc_kl::build_psi(c->kl_variant, c->d_psi + c->psi_off[t], n, p->n_modes, c->d_ma,
                                                    c->d_mb, c->d_psi_tc[t], 0)) &&
                   mlqmc_kl::make_maps(c->kl_variant, c->d_psi_tc[t], mpad, c->d_C, static_cast<int>(ms), p->n_modes,
                                       &c->kl_maps[t]);
        }
        if (!good || !ok(cudaDeviceSynchronize())) {
            free_ctx(c);
            return MLQMC_ERR_CUDA;
        }
        c->kl_tc = true;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    c->pool_budget = std::min<size_t>(free_b / 2, static_cast<size_t>(192) << 30);
    if (!mlqmc_tma::prepare() || !mlqmc_whole::prepare() || !mlqmc_resid::prepare()) {
        free_ctx(c);
        return MLQMC_ERR_CUDA;
    }
    st = tune_smoothers(c);
    if (st == MLQMC_OK) st = tune_kl(c);
    if (st != MLQMC_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return MLQMC_OK;
}

void graph_free(mlqmc_ctx* c);
void round_graphs_free(mlqmc_ctx* c);

extern "C" void mlqmc_destroy(mlqmc_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    graph_free(c);
    free_ctx(c);
}

// ---------------------------------------------------------------------------
// Graph replay of repeated identical calls (fixed-cycle forms, one chunk).
// ---------------------------------------------------------------------------
void graph_reset(mlqmc_ctx* c)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    if (G.exec) {
        cudaStreamSynchronize(G.stream);
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    for (auto& m : G.marks) {
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    G.marks.clear();
    G.seen = 0;
    G.key.clear();
}

void round_graphs_free(mlqmc_ctx* c)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    if (G.stream) cudaStreamSynchronize(G.stream);
    for (auto& e : G.round_execs) cudaGraphExecDestroy(e.exec);
    G.round_execs.clear();
}

void graph_free(mlqmc_ctx* c)
{
    graph_reset(c);
    round_graphs_free(c);
    mlqmc_ctx::GraphCache& G = c->graph;
    if (G.body) cudaStreamDestroy(G.body);
    G.body = nullptr;
    if (G.stream) cudaStreamDestroy(G.stream);
    if (G.in) cudaEventDestroy(G.in);
    if (G.out) cudaEventDestroy(G.out);
    if (G.h_samples) cudaFreeHost(G.h_samples);
    G.stream = nullptr;
    G.in = G.out = nullptr;
    G.h_samples = nullptr;
}

mlqmc_status graph_replay(mlqmc_ctx* c, cudaStream_t st)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    if (!ok(cudaEventRecord(G.in, st)) || !ok(cudaStreamWaitEvent(G.stream, G.in, 0)) ||
        !ok(cudaGraphLaunch(G.exec, G.stream)) || !ok(cudaEventRecord(G.out, G.stream)) ||
        !ok(cudaStreamWaitEvent(st, G.out, 0)))
        return MLQMC_ERR_CUDA;
    c->launches += G.launches;
    ++G.replays;
    if (c->profiling && G.profiled && !G.marks.empty()) {
        // the graph re-records its events on every replay: read them now
        if (!ok(cudaEventSynchronize(G.marks.back().b))) return MLQMC_ERR_CUDA;
        for (const auto& m : G.marks) {
            float ms = 0.0f;
            if (!ok(cudaEventElapsedTime(&ms, m.a, m.b))) return MLQMC_ERR_CUDA;
            c->prof[m.kind][m.level].ms += ms;
            c->prof[m.kind][m.level].n += m.nk;
        }
        for (int k = 0; k < kProfKinds; ++k)
            for (int l = 0; l < kProfLevels; ++l) {
                ProfCell& pc = c->prof[k][l];
                const ProfCell& gw = G.work[k][l];
                pc.bytes += gw.bytes;
                pc.f64 += gw.f64;
                pc.f32 += gw.f32;
                pc.ftc += gw.ftc;
            }
    }
    return MLQMC_OK;
}

// Capture the chunk (upload of the ranked samples + run_chunk) on the graph
// stream, instantiate it and replay it once for this call.
mlqmc_status graph_capture(mlqmc_ctx* c, int count, const int* Bt, int Lmax, double* d_sums, double* d_F,
                           cudaStream_t st)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    if (!G.stream && !ok(cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking))) return MLQMC_ERR_CUDA;
    if (!G.in && !ok(cudaEventCreateWithFlags(&G.in, cudaEventDisableTiming))) return MLQMC_ERR_CUDA;
    if (!G.out && !ok(cudaEventCreateWithFlags(&G.out, cudaEventDisableTiming))) return MLQMC_ERR_CUDA;
    if (!G.h_samples && !ok(cudaMallocHost(&G.h_samples, c->max_samples * sizeof(SampleDesc)))) {
        G.h_samples = nullptr;
        return MLQMC_ERR_OOM;
    }
    // the graph's upload reads G.h_samples: no replay of an older graph may be in flight
    if (!ok(cudaStreamSynchronize(G.stream))) return MLQMC_ERR_CUDA;
    std::memcpy(G.h_samples, G.key.data(), static_cast<size_t>(count) * sizeof(SampleDesc));
    const size_t marks0 = c->marks.size();
    const int64_t launches0 = c->launches;
    std::vector<ProfCell> w0(&c->prof[0][0], &c->prof[0][0] + kProfKinds * kProfLevels);
    if (!ok(cudaStreamBeginCapture(G.stream, cudaStreamCaptureModeThreadLocal))) return MLQMC_ERR_CUDA;
    G.capturing = true;
    mlqmc_status s = ok(cudaMemcpyAsync(c->d_samples, G.h_samples, count * sizeof(SampleDesc), cudaMemcpyHostToDevice,
                                        G.stream))
                         ? run_chunk(c, count, Bt, Lmax, d_sums, d_F, nullptr, G.stream)
                         : MLQMC_ERR_CUDA;
    G.capturing = false;
    cudaGraph_t graph = nullptr;
    const bool ended = ok(cudaStreamEndCapture(G.stream, &graph));
    // whatever happened, the brackets and work recorded while capturing belong to the graph
    G.marks.assign(c->marks.begin() + static_cast<std::ptrdiff_t>(marks0), c->marks.end());
    c->marks.resize(marks0);
    G.launches = c->launches - launches0;
    c->launches = launches0;
    for (int k = 0; k < kProfKinds; ++k)
        for (int l = 0; l < kProfLevels; ++l) {
            ProfCell& pc = c->prof[k][l];
            const ProfCell& before = w0[static_cast<size_t>(k) * kProfLevels + l];
            ProfCell& gw = G.work[k][l];
            gw.bytes = pc.bytes - before.bytes;
            gw.f64 = pc.f64 - before.f64;
            gw.f32 = pc.f32 - before.f32;
            gw.ftc = pc.ftc - before.ftc;
            pc = before;
        }
    if (s == MLQMC_OK && (!ended || !graph)) s = MLQMC_ERR_CUDA;
    if (s == MLQMC_OK && !ok(cudaGraphInstantiate(&G.exec, graph, 0))) {
        G.exec = nullptr;
        s = MLQMC_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (s != MLQMC_OK) {
        graph_reset(c);
        return s;
    }
    G.seen = 2;
    return graph_replay(c, st);
}

// Everything a round graph needs allocated before its capture (nothing may be
// allocated while capturing): the level pools and the converged forms'
// partial-norm buffer.
mlqmc_status prepare_round(mlqmc_ctx* c, const int* Bt, int Lmax)
{
    for (int t = 0; t <= Lmax; ++t) {
        mlqmc_status s = ensure_pool(c, t, Bt[t]);
        if (s != MLQMC_OK) return s;
    }
    if (c->p.refine_rtol > 0.0) {
        int64_t need = 0;
        for (int t = 1; t <= Lmax; ++t) {
            const int64_t n = c->p.coarse_cells << t;
            need = std::max<int64_t>(need, static_cast<int64_t>(Bt[t]) * std::max<int64_t>(1, n * n / 8192));
        }
        if (need > c->part_cap) {
            cudaDeviceSynchronize();
            cudaFree(c->d_part);
            c->d_part = nullptr;
            c->part_cap = 0;
            if (!ok(cudaMalloc(&c->d_part, sizeof(double) * static_cast<size_t>(need)))) return MLQMC_ERR_OOM;
            c->part_cap = need;
        }
    }
    return MLQMC_OK;
}

// One call (one chunk, descriptors already staged) as one graph launch:
// capture run_chunk on the graph stream (converged forms: device-side
// refinement loops), update the instantiated graph of the same launch shape
// in place, or instantiate one, and launch it between events of `st`.
mlqmc_status round_graph(mlqmc_ctx* c, int count, const int* Bt, int Lmax, double* d_sums, double* d_F,
                         cudaStream_t st)
{
    mlqmc_ctx::GraphCache& G = c->graph;
    if (!G.stream && !ok(cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking))) return MLQMC_ERR_CUDA;
    if (!G.body && !ok(cudaStreamCreateWithFlags(&G.body, cudaStreamNonBlocking))) return MLQMC_ERR_CUDA;
    if (!G.in && !ok(cudaEventCreateWithFlags(&G.in, cudaEventDisableTiming))) return MLQMC_ERR_CUDA;
    if (!G.out && !ok(cudaEventCreateWithFlags(&G.out, cudaEventDisableTiming))) return MLQMC_ERR_CUDA;
    // launch shape: the levels that run and their smoothers, the outputs asked for
    std::vector<int32_t> key;
    key.push_back(Lmax);
    for (int t = 0; t <= Lmax; ++t) {
        key.push_back(Bt[t] > 0 ? smoother_for(c, t, Bt[t]) : -1);
        key.push_back(Bt[t] > 0 ? kl_nt_for(c, t, Bt[t]) : 0);
    }
    key.push_back(d_F ? 1 : 0);
    key.push_back(d_sums ? 1 : 0);
    // an instantiated graph may still be running the previous call
    if (!ok(cudaStreamSynchronize(G.stream))) return MLQMC_ERR_CUDA;
    if (!ok(cudaStreamBeginCapture(G.stream, cudaStreamCaptureModeThreadLocal))) return MLQMC_ERR_CUDA;
    G.capturing = true;
    G.round_capture = true;
    mlqmc_status s = run_chunk(c, count, Bt, Lmax, d_sums, d_F, nullptr, G.stream);
    G.capturing = false;
    G.round_capture = false;
    G.in_body = false;
    cudaGraph_t graph = nullptr;
    const bool ended = ok(cudaStreamEndCapture(G.stream, &graph));
    if (s == MLQMC_OK && (!ended || !graph)) s = MLQMC_ERR_CUDA;
    cudaGraphExec_t exec = nullptr;
    if (s == MLQMC_OK) {
        auto it = std::find_if(G.round_execs.begin(), G.round_execs.end(),
                               [&](const mlqmc_ctx::GraphCache::RoundExec& e) { return e.key == key; });
        if (it != G.round_execs.end()) {
            cudaGraphExecUpdateResultInfo info{};
            if (ok(cudaGraphExecUpdate(it->exec, graph, &info))) {
                exec = it->exec;
                ++G.round_updates;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(it->exec);
                G.round_execs.erase(it);
            }
        }
        if (!exec) {
            if (ok(cudaGraphInstantiate(&exec, graph, 0))) {
                ++G.round_instantiations;
                if (G.round_execs.size() >= 16) {
                    cudaGraphExecDestroy(G.round_execs.front().exec);
                    G.round_execs.erase(G.round_execs.begin());
                }
                G.round_execs.push_back({key, exec});
            } else {
                exec = nullptr;
                s = MLQMC_ERR_CUDA;
            }
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (s != MLQMC_OK) return s;
    if (!ok(cudaEventRecord(G.in, st)) || !ok(cudaStreamWaitEvent(G.stream, G.in, 0)) ||
        !ok(cudaGraphLaunch(exec, G.stream)) || !ok(cudaEventRecord(G.out, G.stream)) ||
        !ok(cudaStreamWaitEvent(st, G.out, 0)))
        return MLQMC_ERR_CUDA;
    ++G.round_launches;
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_sample_levels(mlqmc_ctx* c, const mlqmc_work* work, int32_t n_work, double* d_sums,
                                            double* d_F, void* stream)
{
    if (!c || n_work < 0 || (n_work > 0 && !work) || !d_sums) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const mlqmc_problem& p = c->p;
    int64_t total = 0;
    for (int i = 0; i < n_work; ++i) {
        const mlqmc_work& w = work[i];
        if (w.level < 0 || w.level >= p.n_levels || w.n_begin < 0 || w.n_end < w.n_begin || w.r_begin < 0 ||
            w.r_end < w.r_begin || w.r_end > p.n_shifts)
            return MLQMC_ERR_INVALID_ARG;
        if (p.sampler == MLQMC_SAMPLER_LATTICE && p.log2_nmax < 32 && w.n_end > (int64_t(1) << p.log2_nmax))
            return MLQMC_ERR_POINTS_EXHAUSTED;
        if (p.sampler == MLQMC_SAMPLER_MC && w.n_end > (int64_t(1) << 32)) return MLQMC_ERR_POINTS_EXHAUSTED;
        total += (w.n_end - w.n_begin) * (w.r_end - w.r_begin);
    }
    if (total == 0) return MLQMC_OK;
    // expand in work order, then rank by finest level (stable, descending)
    std::vector<SampleDesc> all;
    all.reserve(static_cast<size_t>(total));
    for (int i = 0; i < n_work; ++i) {
        const mlqmc_work& w = work[i];
        for (int r = w.r_begin; r < w.r_end; ++r)
            for (int64_t n = w.n_begin; n < w.n_end; ++n) {
                SampleDesc d;
                d.n = n;
                d.gidx = static_cast<int64_t>(all.size());
                d.r = r;
                d.level = w.level;
                d.canon = 0;
                d.pad = 0;
                all.push_back(d);
            }
    }
    std::stable_sort(all.begin(), all.end(), [](const SampleDesc& x, const SampleDesc& y) { return x.level > y.level; });
    // chunks: consecutive ranks that fit max_samples, the pool budget and the
    // 32-bit flat loops (samples x elements of every level below 2^31)
    std::vector<size_t> lvl_bytes(p.n_levels);
    std::vector<uint64_t> lvl_elems(p.n_levels);
    for (int t = 0; t < p.n_levels; ++t) {
        lvl_bytes[t] = level_bytes_per_sample(p, c->Ka, t);
        lvl_elems[t] = level_elems_per_sample(p, c->Ka, t);
    }
    // graph replay: one chunk, fixed cycles (no host-side convergence loop)
    const bool graphable = c->graph.enabled && p.refine_rtol == 0.0;
    size_t a = 0;
    while (a < all.size()) {
        size_t b = a, bytes = 0;
        uint64_t cnt[MLQMC_MAX_LEVELS] = {};
        while (b < all.size() && static_cast<int64_t>(b - a) < c->max_samples) {
            size_t add = 0;
            bool fits = true;
            for (int t = 0; t <= all[b].level; ++t) {
                add += lvl_bytes[t];
                fits = fits && (cnt[t] + 1) * lvl_elems[t] < (uint64_t(1) << 31);
            }
            if (b > a && (bytes + add > c->pool_budget || !fits)) break;
            bytes += add;
            for (int t = 0; t <= all[b].level; ++t) ++cnt[t];
            ++b;
        }
        const int count = static_cast<int>(b - a);
        for (int q = 0; q < count; ++q) all[a + q].canon = q;
        int Bt[MLQMC_MAX_LEVELS], Lmax = -1;
        count_levels(all.data() + a, count, p.n_levels, Bt, &Lmax);
        {
            const mlqmc_status qs = ensure_qpart(c, Bt, Lmax);
            if (qs != MLQMC_OK) return qs;
        }
        const bool single = a == 0 && b == all.size();
        mlqmc_ctx::GraphCache& G = c->graph;
        if (graphable && single) {
            const bool same = G.seen > 0 && G.epoch == c->pool_epoch && G.sums == d_sums && G.F == d_F &&
                              G.profiled == c->profiling && G.key.size() == all.size() &&
                              std::memcmp(G.key.data(), all.data(), all.size() * sizeof(SampleDesc)) == 0;
            bool fits = true;
            for (int t = 0; t <= Lmax; ++t) fits = fits && Bt[t] <= c->pools[t].cap;
            if (same && G.seen == 2) return graph_replay(c, st);
            if (same && G.seen == 1 && fits) return graph_capture(c, count, Bt, Lmax, d_sums, d_F, st);
        }
        if (graphable && single) graph_reset(c);
        // a call that is not a repeat (an adaptive round): one graph launch
        const bool round = G.enabled && single && !c->profiling &&
                           (G.rounds == 1 || (G.rounds == 2 && p.refine_rtol > 0.0));
        mlqmc_status s = round ? prepare_round(c, Bt, Lmax) : MLQMC_OK;
        if (s == MLQMC_OK) s = stage_samples(c, all.data() + a, count, st);
        if (s != MLQMC_OK) return s;
        s = round ? round_graph(c, count, Bt, Lmax, d_sums, d_F, st)
                  : run_chunk(c, count, Bt, Lmax, d_sums, d_F, nullptr, st);
        if (s != MLQMC_OK) return s;
        if (graphable && single) {  // remember the call: the next identical one is captured
            G.key = all;
            G.sums = d_sums;
            G.F = d_F;
            G.profiled = c->profiling;
            G.epoch = c->pool_epoch;
            G.seen = 1;
        }
        a = b;
    }
    return MLQMC_OK;
}

// Deferred status bits -> the status a call reports (the most severe first).
static mlqmc_status status_of_bits(int h)
{
    if (h & kStatusTimeout) return MLQMC_ERR_TIMEOUT;
    if (h & kStatusNotConverged) return MLQMC_ERR_NOT_CONVERGED;
    if (h & kStatusCheck) return MLQMC_ERR_DEVICE_STATUS;
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_get_device_status(mlqmc_ctx* c, void* stream)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    if (!ok(cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !ok(cudaStreamSynchronize(st)) || !ok(cudaMemsetAsync(c->d_status, 0, sizeof(int), st)) ||
        !ok(cudaStreamSynchronize(st)))
        return MLQMC_ERR_CUDA;
    h |= c->host_status;
    c->host_status = 0;
    return status_of_bits(h);
}

namespace mlqmc {
mlqmc_status fetch_round(mlqmc_ctx* c, const double* d_sums, double* h_sums, size_t n, cudaStream_t st)
{
    if (!c || (n > 0 && (!d_sums || !h_sums))) return MLQMC_ERR_INVALID_ARG;
    if ((n > 0 && !ok(cudaMemcpyAsync(h_sums, d_sums, n * sizeof(double), cudaMemcpyDeviceToHost, st))) ||
        !ok(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !ok(cudaMemsetAsync(c->d_status, 0, sizeof(int), st)) || !ok(cudaStreamSynchronize(st)))
        return MLQMC_ERR_CUDA;
    const int h = *c->h_status | c->host_status;
    c->host_status = 0;
    return status_of_bits(h);
}
}  // namespace mlqmc

extern "C" mlqmc_status mlqmc_modes(const mlqmc_ctx* c, int32_t* a, int32_t* b, double* theta)
{
    if (!c || !a || !b || !theta) return MLQMC_ERR_INVALID_ARG;
    for (int m = 0; m < c->p.n_modes; ++m) {
        a[m] = c->modes.a[m];
        b[m] = c->modes.b[m];
        theta[m] = c->modes.theta[m];
    }
    return MLQMC_OK;
}

namespace {
// A block of `count` samples (level, r, n_begin + i) staged in rank order.
mlqmc_status stage_block(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n_begin, int32_t count, cudaStream_t st,
                         bool check_points = true)
{
    const mlqmc_problem& p = c->p;
    if (level < 0 || level >= p.n_levels || r < 0 || r >= p.n_shifts || n_begin < 0 || count < 0 ||
        count > c->max_samples)
        return MLQMC_ERR_INVALID_ARG;
    if (check_points && p.sampler == MLQMC_SAMPLER_LATTICE && p.log2_nmax < 32 &&
        n_begin + count > (int64_t(1) << p.log2_nmax))
        return MLQMC_ERR_POINTS_EXHAUSTED;
    std::vector<SampleDesc> v(count);
    for (int i = 0; i < count; ++i) {
        v[i].n = n_begin + i;
        v[i].gidx = i;
        v[i].r = r;
        v[i].level = level;
        v[i].canon = i;
        v[i].pad = 0;
    }
    return stage_samples(c, v.data(), count, st);
}
}  // namespace

extern "C" mlqmc_status mlqmc_point_bits(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n_begin, int32_t count,
                                         uint64_t* d_bits, void* stream)
{
    if (!c || !d_bits) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, level, r, n_begin, count, st);
    if (s != MLQMC_OK || count == 0) return s;
    return launch_points(c, c->d_samples, count, nullptr, d_bits, st);
}

extern "C" mlqmc_status mlqmc_normals(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n_begin, int32_t count,
                                      double* d_y, void* stream)
{
    if (!c || !d_y) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, level, r, n_begin, count, st);
    if (s != MLQMC_OK || count == 0) return s;
    return launch_points(c, c->d_samples, count, d_y, nullptr, st);
}

extern "C" mlqmc_status mlqmc_fields(mlqmc_ctx* c, int32_t t, const double* d_y, int32_t count, double* d_k,
                                     void* stream)
{
    if (!c || !d_y || !d_k || t < 0 || t >= c->p.n_levels || count < 0 || count > c->max_samples ||
        static_cast<uint64_t>(count) * level_elems_per_sample(c->p, c->Ka, t) >= (uint64_t(1) << 31))
        return MLQMC_ERR_INVALID_ARG;
    if (count == 0) return MLQMC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, t, 0, 0, count, st, false);
    if (s != MLQMC_OK) return s;
    if (!ok(cudaMemcpyAsync(c->d_Y, d_y, static_cast<size_t>(count) * c->p.n_modes * sizeof(double),
                            cudaMemcpyDeviceToDevice, st)))
        return MLQMC_ERR_CUDA;
    s = ensure_pool(c, t, count);
    if (s != MLQMC_OK) return s;
    s = build_c(c, count, st);
    if (s != MLQMC_OK) return s;
    FmgArgs A = base_args(c);
    s = is_mixed(c->p) ? synth_batched<float>(c, A, t, count, st) : synth_batched<double>(c, A, t, count, st);
    if (s != MLQMC_OK) return s;
    const int64_t n = c->p.coarse_cells << t;
    Timed tm(c, kProfReduce, st, work_of<double>(count * (8.0 + (is_mixed(c->p) ? 4.0 : 8.0)) * n * n, 0.0));
    if (is_mixed(c->p)) kb_k_out<float><<<grid_for(c, count * n * n), 256, 0, st>>>(A, t, count, d_k);
    else kb_k_out<double><<<grid_for(c, count * n * n), 256, 0, st>>>(A, t, count, d_k);
    return last_error();
}

extern "C" mlqmc_status mlqmc_sample_solution(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n, double* d_u,
                                              double* d_F, void* stream)
{
    if (!c || !d_u || !d_F) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, level, r, n, 1, st);
    if (s != MLQMC_OK) return s;
    int Bt[MLQMC_MAX_LEVELS];
    for (int t = 0; t < c->p.n_levels; ++t) Bt[t] = t <= level ? 1 : 0;
    s = ensure_qpart(c, Bt, level);
    if (s != MLQMC_OK) return s;
    s = run_chunk(c, 1, Bt, level, nullptr, nullptr, d_u, st);
    if (s != MLQMC_OK) return s;
    if (!ok(cudaMemcpyAsync(d_F, c->d_F, (level + 1) * sizeof(double), cudaMemcpyDeviceToDevice, st)))
        return MLQMC_ERR_CUDA;
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_profile(mlqmc_ctx* c, int32_t enable)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    for (auto& m : c->marks) {
        cudaEventSynchronize(m.b);
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    c->marks.clear();
    c->profiling = enable != 0;
    for (auto& row : c->prof)
        for (auto& pc : row) pc = ProfCell();
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_profile_work(mlqmc_ctx* c, double* out_bytes, double* out_f64, double* out_f32,
                                           double* out_ftc)
{
    if (!c || !out_bytes || !out_f64 || !out_f32 || !out_ftc) return MLQMC_ERR_INVALID_ARG;
    for (int i = 0; i < kProfKinds; ++i) {
        out_bytes[i] = out_f64[i] = out_f32[i] = out_ftc[i] = 0.0;
        for (const ProfCell& pc : c->prof[i]) {
            out_bytes[i] += pc.bytes;
            out_f64[i] += pc.f64;
            out_f32[i] += pc.f32;
            out_ftc[i] += pc.ftc;
        }
    }
    return MLQMC_OK;
}

namespace {
// Fold the recorded brackets into the per-kind, per-level times (waits for them).
mlqmc_status drain_marks(mlqmc_ctx* c)
{
    for (auto& m : c->marks) {
        if (!ok(cudaEventSynchronize(m.b))) return MLQMC_ERR_CUDA;
        float ms = 0.0f;
        if (!ok(cudaEventElapsedTime(&ms, m.a, m.b))) return MLQMC_ERR_CUDA;
        c->prof[m.kind][m.level].ms += ms;
        c->prof[m.kind][m.level].n += m.nk;
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    c->marks.clear();
    return MLQMC_OK;
}
}  // namespace

extern "C" mlqmc_status mlqmc_profile_read(mlqmc_ctx* c, double* out_ms, int64_t* out_n)
{
    if (!c || !out_ms || !out_n) return MLQMC_ERR_INVALID_ARG;
    const mlqmc_status s = drain_marks(c);
    if (s != MLQMC_OK) return s;
    for (int i = 0; i < kProfKinds; ++i) {
        out_ms[i] = 0.0;
        out_n[i] = 0;
        for (const ProfCell& pc : c->prof[i]) {
            out_ms[i] += pc.ms;
            out_n[i] += pc.n;
        }
    }
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_profile_read_levels(mlqmc_ctx* c, double* out_ms, int64_t* out_n, double* out_bytes,
                                                  double* out_f64, double* out_f32, double* out_ftc)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    const mlqmc_status s = drain_marks(c);
    if (s != MLQMC_OK) return s;
    for (int k = 0; k < kProfKinds; ++k)
        for (int l = 0; l < kProfLevels; ++l) {
            const ProfCell& pc = c->prof[k][l];
            const size_t i = static_cast<size_t>(k) * kProfLevels + l;
            if (out_ms) out_ms[i] = pc.ms;
            if (out_n) out_n[i] = pc.n;
            if (out_bytes) out_bytes[i] = pc.bytes;
            if (out_f64) out_f64[i] = pc.f64;
            if (out_f32) out_f32[i] = pc.f32;
            if (out_ftc) out_ftc[i] = pc.ftc;
        }
    return MLQMC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free FMG from given fields (mlqmc_fmg_fields_noalloc).
// Scratch lives in one static device array; host code reaches it only through
// the address cudaGetSymbolAddress returns (the symbol itself is a host-side
// stand-in, not a device address).
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MLQMC_NOALLOC_SLOTS * size_t(MLQMC_NOALLOC_SLOT_BYTES)];

// Faces and inverse diagonal of one level from k already in L.k.
__device__ void noalloc_faces(const Lv<double>& L)
{
    const int n = L.n;
    for (int idx = threadIdx.x; idx < n * (n + 1); idx += blockDim.x) {
        const int i2 = idx / (n + 1);
        L.kx[i2 * kx_pitch(n) + idx - i2 * (n + 1)] = face_x(L.k, n, i2, idx - i2 * (n + 1));
        const int g = idx / n;
        L.ky[idx] = face_y(L.k, n, g, idx - g * n);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n;
        L.idiag[p] = inv_diag(L.kx, L.ky, n, p - i2 * n, i2);
    }
    __syncthreads();
}

// One CTA per scratch slot; CTA b solves samples b, b + gridDim.x, ...
__global__ void __launch_bounds__(256) k_fmg_noalloc(FmgArgs A, const double* __restrict__ k_in, size_t k_stride,
                                                     int count, double* __restrict__ F_out)
{
    extern __shared__ double smem[];
    const int N0 = A.n0 * A.n0;
    double* Lb = smem;
    double* tmp = Lb + N0 * (A.n0 + 1);
    double* red = tmp + N0;
    double* Fv = red + 40;
    const int slot = blockIdx.x;
    const int Lf = A.n_levels - 1;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const double* ks = k_in + static_cast<size_t>(q) * k_stride;
        for (int t = 0; t <= Lf; ++t) {
            const Lv<double> L = view<double>(A, t, slot);
            for (int p = threadIdx.x; p < L.n * L.n; p += blockDim.x) L.k[p] = ks[p];
            ks += static_cast<size_t>(L.n) * L.n;
            __syncthreads();
            noalloc_faces(L);
        }
        const BlockTeam tm;
        const Lv<double> L0 = view<double>(A, 0, slot);
        chol_factor(tm, Lb, A.n0, L0.kx, L0.ky);
        chol_solve<double, double>(tm, Lb, A.n0, nullptr, L0.u, tmp);
        const double F0 = qoi(tm, L0.u, A.n0, A.qoi, red);
        if (threadIdx.x == 0) Fv[0] = F0;
        for (int t = 1; t <= Lf; ++t) {
            const Lv<double> L = view<double>(A, t, slot);
            const Lv<double> Lc = view<double>(A, t - 1, slot);
            prolong<double, double, false>(tm, Lc.u, Lc.n, L.u);
            for (int m = 0; m < A.mu0; ++m) vcycle<double>(tm, A, slot, t, nullptr, Lb, tmp);
            const double Ft = qoi(tm, L.u, L.n, A.qoi, red);
            if (threadIdx.x == 0) Fv[t] = Ft;
        }
        __syncthreads();
        if (threadIdx.x <= Lf) F_out[static_cast<size_t>(q) * A.n_levels + threadIdx.x] = Fv[threadIdx.x];
        __syncthreads();
    }
}

// Device address of the static scratch, looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

}  // namespace

extern "C" mlqmc_status mlqmc_fmg_fields_noalloc(int32_t coarse_cells, int32_t n_levels, int32_t qoi_kind,
                                                 int32_t mu0, int32_t nu1, int32_t nu2, int32_t count,
                                                 const double* d_k, double* d_F, void* stream)
{
    if (coarse_cells < 2 || (coarse_cells & 1) || n_levels < 1 || count < 0 || !d_k || !d_F || mu0 < 1 ||
        nu1 < 0 || nu2 < 0 || mu0 > 64 || nu1 > 64 || nu2 > 64 ||
        (qoi_kind != MLQMC_QOI_CENTER && qoi_kind != MLQMC_QOI_MEAN))
        return MLQMC_ERR_INVALID_ARG;
    if (coarse_cells > 16 || n_levels > 7 ||
        (static_cast<int64_t>(coarse_cells) << (n_levels - 1)) > MLQMC_NOALLOC_MAX_CELLS)
        return MLQMC_ERR_SCRATCH_LIMIT;
    // slot layout: the levels' arrays one after another
    mlqmc_problem p{};
    p.coarse_cells = coarse_cells;
    p.precision = MLQMC_FP64;
    size_t offs[MLQMC_MAX_LEVELS][kPoolArrs];
    size_t off = 0;
    for (int t = 0; t < n_levels; ++t) {
        size_t st[kPoolArrs];
        level_strides(p, 0, t, st);
        st[kG] = 0;
        st[kU2] = 0;
        for (int a = 0; a < kPoolArrs; ++a) {
            offs[t][a] = off;
            off += st[a];
        }
    }
    if (off > static_cast<size_t>(MLQMC_NOALLOC_SLOT_BYTES)) return MLQMC_ERR_SCRATCH_LIMIT;
    if (count == 0) return MLQMC_OK;
    int dev = 0;
    if (!ok(cudaGetDevice(&dev)) || dev < 0 || dev >= kMaxDevices) return MLQMC_ERR_CUDA;
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            if (!ok(cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) || !ptr) return MLQMC_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    FmgArgs A;
    std::memset(&A, 0, sizeof(A));
    A.n0 = coarse_cells;
    A.n_levels = n_levels;
    A.qoi = qoi_kind;
    A.mu0 = mu0;
    A.nu1 = nu1;
    A.nu2 = nu2;
    for (int t = 0; t < n_levels; ++t) {
        LevelDesc& d = A.lv[t];
        d.n = coarse_cells << t;
        set_divisors(d, A.Ka);
        ArrDesc* arr[kPoolArrs] = {&d.u, &d.bc, &d.kx, &d.ky, &d.idiag, &d.k, &d.G, &d.u64, &d.u2};
        for (int a = 0; a < kPoolArrs; ++a) {
            arr[a]->base = scratch + offs[t][a];
            arr[a]->stride = MLQMC_NOALLOC_SLOT_BYTES;
        }
    }
    size_t k_stride = 0;
    for (int t = 0; t < n_levels; ++t) k_stride += static_cast<size_t>(A.lv[t].n) * A.lv[t].n;
    const size_t N0 = static_cast<size_t>(coarse_cells) * coarse_cells;
    const size_t smem = sizeof(double) * (N0 * (coarse_cells + 1) + N0 + 40 + 16);
    const int grid = std::min<int>(count, MLQMC_NOALLOC_SLOTS);
    k_fmg_noalloc<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(A, d_k, k_stride, count, d_F);
    return ok(cudaGetLastError()) ? MLQMC_OK : MLQMC_ERR_CUDA;
}

extern "C" mlqmc_status mlqmc_last_iterations(mlqmc_ctx* c, int32_t* out)
{
    if (!c || !out) return MLQMC_ERR_INVALID_ARG;
    // device-side loops (round graphs) keep their maxima on the device
    int dev[MLQMC_MAX_LEVELS] = {};
    if (!ok(cudaDeviceSynchronize()) ||
        !ok(cudaMemcpy(dev, c->d_iters + MLQMC_MAX_LEVELS, sizeof(dev), cudaMemcpyDeviceToHost)) ||
        !ok(cudaMemset(c->d_iters + MLQMC_MAX_LEVELS, 0, sizeof(dev))))
        return MLQMC_ERR_CUDA;
    for (int t = 0; t < c->p.n_levels; ++t) {
        out[t] = std::max(c->last_iters[t], dev[t]);
        c->last_iters[t] = 0;
    }
    return MLQMC_OK;
}

extern "C" int64_t mlqmc_launch_count(const mlqmc_ctx* c)
{
    return c ? c->launches : 0;
}

extern "C" mlqmc_status mlqmc_smoother_info(const mlqmc_ctx* c, int32_t* kind, double* tuned_ms)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    for (int t = 0; t < c->p.n_levels; ++t) {
        if (kind) kind[t] = t == 0 ? 0 : c->smoother[t];
        for (int k = 0; k < 5 && tuned_ms; ++k) tuned_ms[t * 5 + k] = c->tune_ms[t][k];
    }
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_schedule_info(const mlqmc_ctx* c, int32_t* smoother_small, double* tuned_small_ms,
                                            int32_t* kl_nt, double* tuned_kl_ms)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    for (int t = 0; t < c->p.n_levels; ++t) {
        if (smoother_small) smoother_small[t] = t == 0 ? 0 : c->smoother_small[t];
        for (int k = 0; k < 5 && tuned_small_ms; ++k) tuned_small_ms[t * 5 + k] = c->tune_small_ms[t][k];
        for (int cls = 0; cls < 2; ++cls) {
            if (kl_nt) kl_nt[t * 2 + cls] = c->d_psi_tc[t] ? c->kl_nt[t][cls] : 0;
            for (int k = 0; k < 2 && tuned_kl_ms; ++k) tuned_kl_ms[(t * 2 + cls) * 2 + k] = c->tune_kl_ms[t][cls][k];
        }
    }
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_set_smoother(mlqmc_ctx* c, int32_t level, int32_t kind)
{
    if (!c || level < 1 || level >= c->p.n_levels || kind < MLQMC_SMOOTHER_GS || kind > MLQMC_SMOOTHER_WHOLE ||
        (kind == MLQMC_SMOOTHER_GS && is_mixed(c->p)) || !smoother_fits(c, kind, level))
        return MLQMC_ERR_INVALID_ARG;
    c->smoother[level] = c->smoother_small[level] = kind;  // every batch size
    ++c->pool_epoch;  // a captured graph runs the old smoother
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_set_graphs(mlqmc_ctx* c, int32_t enable)
{
    if (!c) return MLQMC_ERR_INVALID_ARG;
    if (!enable) {
        graph_reset(c);
        round_graphs_free(c);
    }
    c->graph.enabled = enable != 0;
    return MLQMC_OK;
}

namespace {
// Waits (thread 0) on an mbarrier that nothing arrives on, with the bounded
// wait of the TMA-fed kernels and a limit of limit_ns; the give-up records
// the timeout bit in the context's status word. No copy is issued.
__global__ void k_wait_nothing(int* status, uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mlqmc_ptx::mbar_init(&bar, 1);
        mlqmc_ptx::mbar_init_fence();
        mlqmc_ptx::mbar_wait(&bar, 0, status, kStatusTimeout, limit_ns);
    }
}
}  // namespace

extern "C" mlqmc_status mlqmc_test_wait_timeout(mlqmc_ctx* c, int64_t limit_ns, void* stream)
{
    if (!c || limit_ns < 0 || limit_ns > 100000000) return MLQMC_ERR_INVALID_ARG;
    k_wait_nothing<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(c->d_status, static_cast<uint64_t>(limit_ns));
    return last_error();
}

extern "C" mlqmc_status mlqmc_set_round_graphs(mlqmc_ctx* c, int32_t mode)
{
    if (!c || mode < 0 || mode > 2) return MLQMC_ERR_INVALID_ARG;
    c->graph.rounds = mode;
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_graph_stats(const mlqmc_ctx* c, int64_t* out)
{
    if (!c || !out) return MLQMC_ERR_INVALID_ARG;
    out[0] = c->graph.replays;
    out[1] = c->graph.round_launches;
    out[2] = c->graph.round_updates;
    out[3] = c->graph.round_instantiations;
    return MLQMC_OK;
}

extern "C" int64_t mlqmc_graph_replays(const mlqmc_ctx* c)
{
    return c ? c->graph.replays : 0;
}
