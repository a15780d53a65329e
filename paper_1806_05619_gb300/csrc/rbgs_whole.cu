// Whole-sample red-black smoother for the small levels of the FP32 V-cycles
// (Sec. 4).
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

#include "ptx_async.cuh"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

// Per-sample shared layout (floats): u (n x n), x faces (n rows of pitch n + 4),
// y faces ((n + 1) x n), b (n x n), coarse solution (n/2 x n/2); every part a
// multiple of 4 floats, so every bulk copy starts on a 16-byte boundary.
template <int N>
struct WGeom {
    static constexpr int TS = N <= 32 ? 32 : 256;              // threads per sample
    static constexpr int SPC = N <= 16 ? 8 : (N == 32 ? 4 : 1);  // samples per CTA
    static constexpr int XP = N + 4;                            // kx_pitch(N)
    static constexpr int NC = N / 2;
    static constexpr int oU = 0;
    static constexpr int oKX = oU + N * N;
    static constexpr int oKY = oKX + N * XP;
    static constexpr int oB = oKY + (N + 1) * N;
    static constexpr int oE = oB + N * N;
    static constexpr int per = oE + NC * NC;
    static constexpr size_t bytes = 128 + sizeof(float) * static_cast<size_t>(SPC) * per;
    static_assert(N % 8 == 0 && per % 4 == 0 && SPC * 8 <= 128, "16-byte aligned parts, barrier area");
};

template <int N>
__device__ __forceinline__ void team_sync()
{
    if constexpr (WGeom<N>::TS == 32) __syncwarp();
    else __syncthreads();
}

template <int N, bool PRE, bool POST>
__global__ void __launch_bounds__(WGeom<N>::TS * WGeom<N>::SPC)
    kb_rbgs_whole(FmgArgs A, int t, int B, int ns, int ones, int first)
{
    using Gm = WGeom<N>;
    constexpr int TS = Gm::TS, NC = Gm::NC, XP = Gm::XP;
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
    const int g = threadIdx.x / TS;
    const int ts = threadIdx.x - g * TS;
    const int i = blockIdx.x * Gm::SPC + g;
    // uniform per team (a warp, or the CTA when SPC = 1): the team barriers below stay uniform
    const bool act = i < B && !(A.active && !A.active[i]);
    float* S = reinterpret_cast<float*>(smraw + 128) + g * Gm::per;
    if (threadIdx.x == 0) {
        for (int s = 0; s < Gm::SPC; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (!act) return;
    const int ic = i;
    float* gu = at<float>(A.lv[t].u, ic);
    if (ts == 0) {
        uint32_t bytes = 4u * (N * N + N * XP + (N + 1) * N + (ones ? 0 : N * N) + (POST ? NC * NC : 0));
        uint64_t* bar = &bars[g];
        mbar_arrive_tx(bar, bytes);
        bulk_load(S + Gm::oU, gu, 4u * N * N, bar);
        bulk_load(S + Gm::oKX, at<float>(A.lv[t].kx, ic), 4u * N * XP, bar);
        bulk_load(S + Gm::oKY, at<float>(A.lv[t].ky, ic), 4u * (N + 1) * N, bar);
        if (!ones) bulk_load(S + Gm::oB, at<float>(A.lv[t].bc, ic), 4u * N * N, bar);
        if (POST) bulk_load(S + Gm::oE, at<float>(A.lv[t - 1].u, ic), 4u * NC * NC, bar);
    }
    if (!mbar_wait(&bars[g], 0, A.status, kStatusTimeout)) {
        // gave up: let the copies land before the team leaves, then skip the work
        const uint64_t t0 = now_ns();
        while (!mbar_test(&bars[g], 0) && now_ns() - t0 < 1000000000ull) {
        }
        return;
    }
    float* su = S + Gm::oU;
    const float* skx = S + Gm::oKX;
    const float* sky = S + Gm::oKY;
    const float* sb = S + Gm::oB;
    if constexpr (POST) {
        // u += P e, one coarse parent (2 x 2 fine cells) per step: the parent's
        // 3 x 3 neighbourhood, odd reflection across the boundary (prolong_cell's arithmetic)
        const float* se = S + Gm::oE;
        for (int q = ts; q < NC * NC; q += TS) {
            const int I2 = q / NC, I1 = q - (q / NC) * NC;
            const bool lo1 = I1 == 0, hi1 = I1 == NC - 1, lo2 = I2 == 0, hi2 = I2 == NC - 1;
            float E[3][3];
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const bool ry = (dy < 0 && lo2) || (dy > 0 && hi2);
                    const bool rx = (dx < 0 && lo1) || (dx > 0 && hi1);
                    const float v = se[(I2 + (ry ? 0 : dy)) * NC + I1 + (rx ? 0 : dx)];
                    E[dy + 1][dx + 1] = (ry != rx) ? -v : v;
                }
            }
            float* f = su + (2 * I2) * N + 2 * I1;
#pragma unroll
            for (int fy = 0; fy < 2; ++fy)
#pragma unroll
                for (int fx = 0; fx < 2; ++fx)
                    f[fy * N + fx] +=
                        fmaf(0.5625f, E[1][1], fmaf(0.1875f, E[1][2 * fx] + E[2 * fy][1], 0.0625f * E[2 * fy][2 * fx]));
        }
        team_sync<N>();
    }
    const float h2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
    for (int ph = 0; ph < 2 * ns; ++ph) {
        const int colour = (first + ph) & 1;
        for (int q = ts; q < N * NC; q += TS) {
            const int y = q / NC;
            const int x = 2 * (q - y * NC) + ((y + colour) & 1);
            const int c0 = y * N + x;
            const float* kr = skx + y * XP;
            const float w = kr[x], e = kr[x + 1];
            const float nn = sky[c0], so = sky[c0 + N];
            float acc = h2 * (ones ? 1.0f : sb[c0]);
            acc += w * (x > 0 ? su[c0 - 1] : 0.0f);
            acc += e * (x < N - 1 ? su[c0 + 1] : 0.0f);
            acc += nn * (y > 0 ? su[c0 - N] : 0.0f);
            acc += so * (y < N - 1 ? su[c0 + N] : 0.0f);
            su[c0] = __fdividef(acc, w + e + nn + so);  // hardware reciprocal: within 2 ulp
        }
        team_sync<N>();
    }
    if constexpr (PRE) {
        // bc of level t-1: mean over the 4 children of b - A u (resid_restrict_cell's arithmetic)
        const float ih2 = static_cast<float>(N) * static_cast<float>(N);
        float* gbc = at<float>(A.lv[t - 1].bc, ic);
        for (int q = ts; q < NC * NC; q += TS) {
            const int I2 = q / NC, I1 = q - (q / NC) * NC;
            float s = 0.0f;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int x = 2 * I1 + (d & 1), y = 2 * I2 + (d >> 1);
                const int c0 = y * N + x;
                const float up = su[c0];
                const float* kr = skx + y * XP;
                float a2 = kr[x] * (up - (x > 0 ? su[c0 - 1] : 0.0f));
                a2 += kr[x + 1] * (up - (x < N - 1 ? su[c0 + 1] : 0.0f));
                a2 += sky[c0] * (up - (y > 0 ? su[c0 - N] : 0.0f));
                a2 += sky[c0 + N] * (up - (y < N - 1 ? su[c0 + N] : 0.0f));
                s += (ones ? 1.0f : sb[c0]) - ih2 * a2;
            }
            gbc[q] = 0.25f * s;
        }
    }
    for (int q = ts; q < N * N / 4; q += TS) reinterpret_cast<float4*>(gu)[q] = reinterpret_cast<const float4*>(su)[q];
}

template <int N, bool PRE, bool POST>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_whole<N, PRE, POST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(WGeom<N>::bytes)) == cudaSuccess;
}

template <int N>
bool attrs()
{
    return attr<N, false, false>() && attr<N, true, false>() && attr<N, false, true>();
}

template <int N>
void go(const FmgArgs& A, int t, int B, int ns, int ones, int first, bool pre, bool post, cudaStream_t st)
{
    using Gm = WGeom<N>;
    const int grid = (B + Gm::SPC - 1) / Gm::SPC;
    const int threads = Gm::TS * Gm::SPC;
    if (pre) kb_rbgs_whole<N, true, false><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first);
    else if (post) kb_rbgs_whole<N, false, true><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first);
    else kb_rbgs_whole<N, false, false><<<grid, threads, Gm::bytes, st>>>(A, t, B, ns, ones, first);
}

}  // namespace

namespace mlqmc_whole {

bool supported(int n)
{
    return n == 8 || n == 16 || n == 32 || n == 64;
}

bool prepare()
{
    return attrs<8>() && attrs<16>() && attrs<32>() && attrs<64>();
}

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool pre, bool post, cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n || ns < 0 || (pre && post)) return false;
    switch (n) {
    case 8: go<8>(A, t, B, ns, ones, first, pre, post, st); break;
    case 16: go<16>(A, t, B, ns, ones, first, pre, post, st); break;
    case 32: go<32>(A, t, B, ns, ones, first, pre, post, st); break;
    default: go<64>(A, t, B, ns, ones, first, pre, post, st); break;
    }
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mlqmc_whole
