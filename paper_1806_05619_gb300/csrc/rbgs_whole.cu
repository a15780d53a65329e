// Whole-sample red-black smoother for the small levels of the V-cycles
// (Sec. 4), FP32 and FP64 (n <= 64).
//
// A sample's whole level (n <= 64) fits in shared memory: one warp (n <= 32,
// several samples per CTA) or one CTA of 256 threads (n = 64) brings u, the
// faces, b and, for the fused correction, the coarse solution with 1D bulk
// copies (the TMA's untiled form), runs the red-black sweeps with only a warp
// (or CTA) barrier between half sweeps, and writes u back in place: no halo
// is read twice and no cell is updated twice per half sweep. The
// pre-smoothing pass also forms the restricted residual (bc of level t-1),
// the post-smoothing pass first adds the coarse-grid correction P e.
#include "rbgs_whole.h"

#include <cstdint>
#include <type_traits>

#include "ptx_async.cuh"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

// Per-sample shared layout (elements of T): u (n x n), x faces (n rows of
// pitch n + 4), y faces ((n + 1) x n), b (n x n), for FP64 1/D (n x n; the
// FP64 form multiplies by the stored reciprocal, as kb_gs does), coarse
// solution (n/2 x n/2); every part a multiple of 16 bytes, so every bulk
// copy starts on a 16-byte boundary.
template <typename T, int N>
struct WGeom {
    static constexpr bool F64 = sizeof(T) == 8;
    static constexpr int TS = N <= 32 ? 32 : 256;  // threads per sample
    static constexpr int SPC = N == 64 ? 1 : (N <= 16 ? 8 : (F64 ? 2 : 4));  // samples per CTA
    static constexpr int XP = N + 4;               // kx_pitch(N)
    static constexpr int NC = N / 2;
    static constexpr int oU = 0;
    static constexpr int oKX = oU + N * N;
    static constexpr int oKY = oKX + N * XP;
    static constexpr int oB = oKY + (N + 1) * N;
    static constexpr int oD = oB + N * N;
    static constexpr int oE = oD + (F64 ? N * N : 0);
    static constexpr int per = oE + NC * NC;
    static constexpr size_t bytes = 128 + sizeof(T) * static_cast<size_t>(SPC) * per;
    static_assert(N % 8 == 0 && (per * sizeof(T)) % 16 == 0 && SPC * 8 <= 128, "16-byte aligned parts, barriers");
};

template <typename T, int N>
__device__ __forceinline__ void team_sync()
{
    if constexpr (WGeom<T, N>::TS == 32) __syncwarp();
    else __syncthreads();
}

template <typename T, int N, bool PRE, bool POST>
__global__ void __launch_bounds__(WGeom<T, N>::TS * WGeom<T, N>::SPC)
    kb_rbgs_whole(FmgArgs A, int t, int B, int ns, int ones, int first, int zin)
{
    using Gm = WGeom<T, N>;
    constexpr uint32_t es = sizeof(T);
    constexpr int TS = Gm::TS, NC = Gm::NC, XP = Gm::XP;
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
    const int g = threadIdx.x / TS;
    const int ts = threadIdx.x - g * TS;
    const int i = blockIdx.x * Gm::SPC + g;
    // uniform per team (a warp, or the CTA when SPC = 1): the team barriers below stay uniform
    const bool act = i < B && !(A.active && !A.active[i]);
    T* S = reinterpret_cast<T*>(smraw + 128) + g * Gm::per;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Gm::SPC; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (!act) return;
    const int ic = i;
    T* gu = at<T>(A.lv[t].u, ic);
    // zin (pre-smoothing of a correction, never with POST): u is zero on entry,
    // so it is not read but cleared in shared memory
    if (ts == 0) {
        uint32_t bytes = es * ((zin ? 0 : N * N) + N * XP + (N + 1) * N + (ones ? 0 : N * N) + (Gm::F64 ? N * N : 0) +
                               (POST ? NC * NC : 0));
        uint64_t* bar = &bars[g];
        mbar_arrive_tx(bar, bytes);
        if (!zin) bulk_load(S + Gm::oU, gu, es * N * N, bar);
        bulk_load(S + Gm::oKX, at<T>(A.lv[t].kx, ic), es * N * XP, bar);
        bulk_load(S + Gm::oKY, at<T>(A.lv[t].ky, ic), es * (N + 1) * N, bar);
        if (!ones) bulk_load(S + Gm::oB, at<T>(A.lv[t].bc, ic), es * N * N, bar);
        if (Gm::F64) bulk_load(S + Gm::oD, at<T>(A.lv[t].idiag, ic), es * N * N, bar);
        if (POST) bulk_load(S + Gm::oE, at<T>(A.lv[t - 1].u, ic), es * NC * NC, bar);
    }
    if (!mbar_wait(&bars[g], 0, A.status, kStatusTimeout)) {
        // gave up: let the copies land before the team leaves, then skip the work
        const uint64_t t0 = now_ns();
        while (!mbar_test(&bars[g], 0) && now_ns() - t0 < 1000000000ull) {
        }
        return;
    }
    T* su = S + Gm::oU;
    if (zin) {
        for (int q = ts; q < N * N; q += TS) su[q] = T(0);
        team_sync<T, N>();
    }
    const T* skx = S + Gm::oKX;
    const T* sky = S + Gm::oKY;
    const T* sb = S + Gm::oB;
    const T* sd = S + Gm::oD;
    if constexpr (POST) {
        // u += P e, one coarse parent (2 x 2 fine cells) per step: the parent's
        // 3 x 3 neighbourhood, odd reflection across the boundary (prolong_cell's arithmetic)
        const T* se = S + Gm::oE;
        for (int q = ts; q < NC * NC; q += TS) {
            const int I2 = q / NC, I1 = q - (q / NC) * NC;
            const bool lo1 = I1 == 0, hi1 = I1 == NC - 1, lo2 = I2 == 0, hi2 = I2 == NC - 1;
            T E[3][3];
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const bool ry = (dy < 0 && lo2) || (dy > 0 && hi2);
                    const bool rx = (dx < 0 && lo1) || (dx > 0 && hi1);
                    const T v = se[(I2 + (ry ? 0 : dy)) * NC + I1 + (rx ? 0 : dx)];
                    E[dy + 1][dx + 1] = (ry != rx) ? -v : v;
                }
            }
            T* f = su + (2 * I2) * N + 2 * I1;
#pragma unroll
            for (int fy = 0; fy < 2; ++fy)
#pragma unroll
                for (int fx = 0; fx < 2; ++fx)
                    f[fy * N + fx] +=
                        fma(T(0.5625), E[1][1], fma(T(0.1875), E[1][2 * fx] + E[2 * fy][1], T(0.0625) * E[2 * fy][2 * fx]));
        }
        team_sync<T, N>();
    }
    const T h2 = T(1) / (T(N) * T(N));
    for (int ph = 0; ph < 2 * ns; ++ph) {
        const int colour = (first + ph) & 1;
        for (int q = ts; q < N * NC; q += TS) {
            // n <= 32: cells row-major; n = 64: each warp slot covers 16 cells
            // of two neighbouring rows (lanes 0-15 and 16-31), whose opposite
            // colour parities put the 32 accesses in 32 distinct banks
            int y, m;
            if constexpr (NC >= 32) {
                constexpr int SEG = NC / 16;  // 16-cell segments per row
                const int unit = q >> 5, lane = q & 31;
                y = 2 * (unit / SEG) + (lane >> 4);
                m = 16 * (unit - (unit / SEG) * SEG) + (lane & 15);
            } else {
                y = q / NC;
                m = q - y * NC;
            }
            const int x = 2 * m + ((y + colour) & 1);
            const int c0 = y * N + x;
            const T* kr = skx + y * XP;
            const T w = kr[x], e = kr[x + 1];
            const T nn = sky[c0], so = sky[c0 + N];
            T acc = h2 * (ones ? T(1) : sb[c0]);
            acc += w * (x > 0 ? su[c0 - 1] : T(0));
            acc += e * (x < N - 1 ? su[c0 + 1] : T(0));
            acc += nn * (y > 0 ? su[c0 - N] : T(0));
            acc += so * (y < N - 1 ? su[c0 + N] : T(0));
            if constexpr (Gm::F64) su[c0] = acc * sd[c0];  // the stored 1/D, as kb_gs
            else su[c0] = __fdividef(acc, w + e + nn + so);  // hardware reciprocal: within 2 ulp
        }
        team_sync<T, N>();
    }
    if constexpr (PRE) {
        // bc of level t-1: mean over the 4 children of b - A u (resid_restrict_cell's arithmetic)
        const T ih2 = T(N) * T(N);
        T* gbc = at<T>(A.lv[t - 1].bc, ic);
        for (int q = ts; q < NC * NC; q += TS) {
            const int I2 = q / NC, I1 = q - (q / NC) * NC;
            T s = T(0);
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int x = 2 * I1 + (d & 1), y = 2 * I2 + (d >> 1);
                const int c0 = y * N + x;
                const T up = su[c0];
                const T* kr = skx + y * XP;
                T a2 = kr[x] * (up - (x > 0 ? su[c0 - 1] : T(0)));
                a2 += kr[x + 1] * (up - (x < N - 1 ? su[c0 + 1] : T(0)));
                a2 += sky[c0] * (up - (y > 0 ? su[c0 - N] : T(0)));
                a2 += sky[c0 + N] * (up - (y < N - 1 ? su[c0 + N] : T(0)));
                s += (ones ? T(1) : sb[c0]) - ih2 * a2;
            }
            gbc[q] = T(0.25) * s;
        }
    }
    using V = typename std::conditional<Gm::F64, double2, float4>::type;  // 16-byte stores
    constexpr int VE = 16 / sizeof(T);
    for (int q = ts; q < N * N / VE; q += TS) reinterpret_cast<V*>(gu)[q] = reinterpret_cast<const V*>(su)[q];
}

template <typename T, int N, bool PRE, bool POST>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_whole<T, N, PRE, POST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(WGeom<T, N>::bytes)) == cudaSuccess;
}

template <typename T, int N>
bool attrs()
{
    return attr<T, N, false, false>() && attr<T, N, true, false>() && attr<T, N, false, true>();
}

template <typename T, int N>
void go(const FmgArgs& A, int t, int B, int ns, int ones, int first, bool pre, bool post, int zin, cudaStream_t st)
{
    using Gm = WGeom<T, N>;
    const int grid = (B + Gm::SPC - 1) / Gm::SPC;
    const int threads = Gm::TS * Gm::SPC;
    if (pre) kb_rbgs_whole<T, N, true, false><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first, zin);
    else if (post) kb_rbgs_whole<T, N, false, true><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first, 0);
    else kb_rbgs_whole<T, N, false, false><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first, zin);
}

}  // namespace

namespace mlqmc_whole {

bool supported(int n, bool fp64)
{
    return n == 8 || n == 16 || n == 32 || n == 64;  // FP64 64 x 64: 171 KB, one sample per CTA
}

bool prepare()
{
    return attrs<float, 8>() && attrs<float, 16>() && attrs<float, 32>() && attrs<float, 64>() &&
           attrs<double, 8>() && attrs<double, 16>() && attrs<double, 32>() && attrs<double, 64>();
}

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool pre, bool post, bool zin, bool fp64,
            cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n, fp64) || t < 1 || A.lv[t].n != n || ns < 0 || (pre && post) || (zin && post)) return false;
    if (fp64) {
        switch (n) {
        case 8: go<double, 8>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        case 16: go<double, 16>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        case 32: go<double, 32>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        default: go<double, 64>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        }
    } else {
        switch (n) {
        case 8: go<float, 8>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        case 16: go<float, 16>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        case 32: go<float, 32>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        default: go<float, 64>(A, t, B, ns, ones, first, pre, post, zin ? 1 : 0, st); break;
        }
    }
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mlqmc_whole
