// Wavefront red-black Gauss-Seidel smoother for the FP32 V-cycles (Sec. 4).
//
// One CTA of 128 threads owns G = 256 / n samples of one level (n cells per
// side, n / 2 threads per sample; thread tp owns the cell pair (2 tp, 2 tp + 1)
// of every row) and streams their grids from the first row to the last. The
// read-only rows (x faces, y faces, right-hand side and, for the fused
// coarse-grid correction, the coarse solution) arrive by bulk copies
// (cp.async.bulk, the TMA's 1D form) into rings in shared memory, one
// mbarrier per ring slot counting a row bundle's bytes; each thread brings
// its own cells of u with cp.async into a u ring that only threads write.
//
// Half sweep k (colour (first + k) & 1, k = 0 .. 2 ns - 1) runs 2k rows behind
// the newest row: at step j it updates row j - 2k. A half sweep then reads
// (rows y - 1, y, y + 1 of the other colour) only values the previous half
// sweep finished in earlier steps, and no row one half sweep writes in a step
// is read by another in that step, so the result is exactly ns red-black
// sweeps and one barrier per step suffices; each step loads all its operands
// first, so the half sweeps' arithmetic overlaps. Finished rows (after the
// last half sweep) are written back in place, so every array is read once and
// u written once per launch. Optional fusions on the same pass: the
// coarse-grid correction u += P e (bilinear, odd reflection) on each row as it
// arrives, and the restricted residual of the finished rows, two fine rows per
// coarse row. Every wait on a barrier is bounded.
#include "rbgs_stream.h"

#include <cstdint>

#include "ptx_async.cuh"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

constexpr int kRing = 16;       // rows kept per array (power of two)
constexpr int kAhead = 4;       // row bundles in flight beyond the next one needed
constexpr int kCoarseRing = 8;  // coarse rows kept for the fused correction
constexpr int kThreads = 128;

// Shared-memory layout of one sample (floats): kRing rows of u, x faces
// (pitch kx_pitch(N)), y faces (face row f in slot f mod kRing), b, then
// kCoarseRing coarse rows. Every row starts on a 16-byte boundary.
template <int N>
struct Geom {
    static constexpr int G = 2 * kThreads / N;  // samples per CTA
    static constexpr int TPS = N / 2;            // threads per sample
    static constexpr int XP = N + 4;             // kx_pitch(N)
    static constexpr int NC = N / 2;             // coarse side
    static constexpr int oU = 0;
    static constexpr int oKX = oU + kRing * N;
    static constexpr int oKY = oKX + kRing * XP;
    static constexpr int oB = oKY + kRing * N;
    static constexpr int oE = oB + kRing * N;
    static constexpr int per = oE + kCoarseRing * NC;
    static constexpr int kBarBytes = 128;  // kRing mbarriers, padded
    static constexpr size_t bytes = kBarBytes + sizeof(float) * static_cast<size_t>(G) * per;
    static_assert(N % 8 == 0 && G * TPS == kThreads, "row copies need 16-byte multiples");
    static_assert((per * sizeof(float)) % 16 == 0 && (XP * sizeof(float)) % 16 == 0, "16-byte aligned rows");
    static_assert(kRing * 8 <= kBarBytes, "barrier area");
};

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int P>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(P) : "memory");
}

// Operands of one red-black update of cell c of row y.
struct Upd {
    float b, w, e, nn, so, uw, ue, un, us;
};

template <int N, int NS, bool PRE, bool POST>
__global__ void __launch_bounds__(kThreads, 3) kb_rbgs_stream(FmgArgs A, int t, int B, int ones, int first)
{
    using Gm = Geom<N>;
    constexpr int LAG = 2 * (2 * NS - 1);  // rows between the first and the last half sweep
    constexpr int M = kRing - 1;
    constexpr int CM = kCoarseRing - 1;
    // a slot is refilled kRing - 2 - kAhead steps after its row arrived; the
    // last reader of a row (the residual, LAG + 2 rows behind) must be done by then
    static_assert(kRing >= kAhead + LAG + 6, "ring too short for the stagger");
    static_assert(kCoarseRing >= 5 && (kCoarseRing & CM) == 0, "coarse ring");
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);

    const int g = threadIdx.x / Gm::TPS;
    const int tp = threadIdx.x - g * Gm::TPS;
    const int i = blockIdx.x * Gm::G + g;
    const bool act = i < B && !(A.active && !A.active[i]);
    const int ic = act ? i : 0;
    float* S = reinterpret_cast<float*>(smraw + Gm::kBarBytes) + g * Gm::per;
    float* sU = S + Gm::oU;
    float* sKX = S + Gm::oKX;
    float* sKY = S + Gm::oKY;
    float* sB = S + Gm::oB;
    float* sE = S + Gm::oE;
    float* gu = at<float>(A.lv[t].u, ic);
    const float* gkx = at<float>(A.lv[t].kx, ic);
    const float* gky = at<float>(A.lv[t].ky, ic);
    const float* gb = at<float>(A.lv[t].bc, ic);
    const float* ge = POST ? at<float>(A.lv[t - 1].u, ic) : nullptr;
    float* gbc = PRE ? at<float>(A.lv[t - 1].bc, ic) : nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) mbar_init(&full[s], Gm::G);
        mbar_init_fence();
    }
    __syncthreads();

    // Bundle r: x faces and b of row r, y face row r + 1 (and face row 0 with
    // r = 0), with the correction coarse row r / 2 + 1 on even r (and coarse
    // row 0 with r = 0). Copy l is issued by thread l mod TPS of the sample,
    // the arrival with the byte count by thread 0.
    auto issue = [&](int r) {
        uint64_t* bar = &full[r & M];
        if (!act) {
            if (tp == 0) mbar_arrive(bar);
            return;
        }
        const int me = (POST && !(r & 1) && (r >> 1) + 1 < Gm::NC) ? (r >> 1) + 1 : -1;
        if (tp == 0) {
            uint32_t bytes = 4u * (N + Gm::XP);
            if (!ones) bytes += 4u * N;
            if (r == 0) bytes += 4u * N;
            if (POST && r == 0) bytes += 4u * Gm::NC;
            if (me >= 0) bytes += 4u * Gm::NC;
            mbar_arrive_tx(bar, bytes);
        }
        for (int l = tp; l < 6; l += Gm::TPS) {
            if (l == 0) bulk_load(sKX + (r & M) * Gm::XP, gkx + static_cast<size_t>(r) * Gm::XP, 4u * Gm::XP, bar);
            else if (l == 1) bulk_load(sKY + ((r + 1) & M) * N, gky + static_cast<size_t>(r + 1) * N, 4u * N, bar);
            else if (l == 2 && !ones) bulk_load(sB + (r & M) * N, gb + static_cast<size_t>(r) * N, 4u * N, bar);
            else if (l == 3 && r == 0) bulk_load(sKY, gky, 4u * N, bar);
            else if (l == 4 && POST && r == 0) bulk_load(sE, ge, 4u * Gm::NC, bar);
            else if (l == 5 && me >= 0)
                bulk_load(sE + (me & CM) * Gm::NC, ge + static_cast<size_t>(me) * Gm::NC, 4u * Gm::NC, bar);
        }
    };
    // own cells of u row r (one cp.async group per row; empty groups keep the count)
    auto fetch_u = [&](int r) {
        if (act && r < N) cp_async8(sU + (r & M) * N + 2 * tp, gu + static_cast<size_t>(r) * N + 2 * tp);
        cp_async_commit();
    };

    bool live = true;
    for (int r = 0; r < kAhead + 2; ++r) {
        if (r < N) issue(r);
        fetch_u(r);
    }

    const float h2 = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
    const float ih2 = static_cast<float>(N) * static_cast<float>(N);
    float racc = 0.0f;
    constexpr int JL = N - 1 + LAG + (PRE ? 2 : 0);
#pragma unroll 1
    for (int j = -2; j <= JL; ++j) {
        const int rn = j + 2 + kAhead;
        if (j >= 0) {
            if (rn < N) issue(rn);
            fetch_u(rn);
        }
        const int ra = j + 2;
        cp_async_wait<kAhead>();  // own cells of u row ra (and older) have landed
        if (ra < N && act && live) live = mbar_wait(&full[ra & M], (ra / kRing) & 1, A.status, kStatusTimeout);
        // every thread reaches the one barrier below (no barrier inside divergent code)
        if (act) {
            // ---- loads: every operand of this step (rows no one writes in this step)
            float2 upost = make_float2(0.f, 0.f);
            float ea0 = 0.f, ea1 = 0.f, eb0 = 0.f, eb1 = 0.f, ec0 = 0.f, ec1 = 0.f;
            int o1m = 0, o2m = 0;
            if (POST && ra < N) {
                const int I2 = ra >> 1;
                const int J2 = (ra & 1) ? I2 + 1 : I2 - 1;
                const bool o2 = J2 < 0 || J2 >= Gm::NC;
                const int K2 = o2 ? I2 : J2;
                const float* ea = sE + (I2 & CM) * Gm::NC;
                const float* ek = sE + (K2 & CM) * Gm::NC;
                // coarse columns tp - 1, tp, tp + 1 of rows I2 and K2 (reflected at the boundary)
                const int L1 = tp > 0 ? tp - 1 : tp, R1 = tp + 1 < Gm::NC ? tp + 1 : tp;
                ea0 = ea[tp];
                ea1 = ea[L1];
                eb0 = ea[R1];
                eb1 = ek[tp];
                ec0 = ek[L1];
                ec1 = ek[R1];
                o1m = (tp > 0 ? 0 : 1) | (tp + 1 < Gm::NC ? 0 : 2);
                o2m = o2 ? 1 : 0;
                upost = *reinterpret_cast<const float2*>(sU + (ra & M) * N + 2 * tp);
            }
            Upd U[2 * NS];
            int cs[2 * NS];
#pragma unroll
            for (int k = 0; k < 2 * NS; ++k) {
                const int y = j - 2 * k;
                const int s = y & M;
                const int c = 2 * tp + ((y + first + k) & 1);
                cs[k] = c;
                if (y < 0 || y >= N) continue;
                const float* ur = sU + s * N;
                const float* kxr = sKX + s * Gm::XP;
                U[k].b = ones ? 1.0f : sB[s * N + c];
                U[k].w = kxr[c];
                U[k].e = kxr[c + 1];
                U[k].nn = sKY[s * N + c];
                U[k].so = sKY[((y + 1) & M) * N + c];
                U[k].uw = c > 0 ? ur[c - 1] : 0.0f;
                U[k].ue = c < N - 1 ? ur[c + 1] : 0.0f;
                U[k].un = y > 0 ? sU[((y - 1) & M) * N + c] : 0.0f;
                U[k].us = y < N - 1 ? sU[((y + 1) & M) * N + c] : 0.0f;
            }
            const int yo = j - LAG;
            float uo_other = 0.0f;  // the cell of the finished row the last half sweep does not touch
            if (yo >= 0 && yo < N) uo_other = sU[(yo & M) * N + (cs[2 * NS - 1] ^ 1)];
            const int yr = j - LAG - 2;
            float ru[2], rw[2], re[2], rn_[2], rs[2], rkw[2], rke[2], rkn[2], rks[2], rb[2];
            if (PRE && yr >= 0 && yr < N) {
                const int s = yr & M;
                const float* ur = sU + s * N;
                const float* kxr = sKX + s * Gm::XP;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 2 * tp + h;
                    ru[h] = ur[c];
                    rw[h] = c > 0 ? ur[c - 1] : 0.0f;
                    re[h] = c < N - 1 ? ur[c + 1] : 0.0f;
                    rn_[h] = yr > 0 ? sU[((yr - 1) & M) * N + c] : 0.0f;
                    rs[h] = yr < N - 1 ? sU[((yr + 1) & M) * N + c] : 0.0f;
                    rkw[h] = kxr[c];
                    rke[h] = kxr[c + 1];
                    rkn[h] = sKY[s * N + c];
                    rks[h] = sKY[((yr + 1) & M) * N + c];
                    rb[h] = ones ? 1.0f : sB[s * N + c];
                }
            }
            // ---- arithmetic and stores
            if (POST && ra < N) {
                // u += P e on the two cells of row ra (same arithmetic as prolong_cell)
                const bool o2 = o2m != 0;
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool o1 = h ? (o1m & 2) != 0 : (o1m & 1) != 0;
                    const float a = ea0;
                    const float b0 = h ? eb0 : ea1;  // row I2, column K1
                    const float c0 = eb1;            // row K2, column I1
                    const float d0 = h ? ec1 : ec0;  // row K2, column K1
                    const float bb = o1 ? -b0 : b0;
                    const float cc = o2 ? -c0 : c0;
                    const float dd = (o1 != o2) ? -d0 : d0;
                    v[h] = fmaf(0.5625f, a, fmaf(0.1875f, bb + cc, 0.0625f * dd));
                }
                *reinterpret_cast<float2*>(sU + (ra & M) * N + 2 * tp) = make_float2(upost.x + v[0], upost.y + v[1]);
            }
            float ulast = 0.0f;
#pragma unroll
            for (int k = 0; k < 2 * NS; ++k) {
                const int y = j - 2 * k;
                if (y < 0 || y >= N) continue;
                const Upd& q = U[k];
                float acc = h2 * q.b;
                acc += q.w * q.uw;
                acc += q.e * q.ue;
                acc += q.nn * q.un;
                acc += q.so * q.us;
                const float v = __fdividef(acc, q.w + q.e + q.nn + q.so);  // hardware reciprocal: within 2 ulp
                sU[(y & M) * N + cs[k]] = v;
                if (k == 2 * NS - 1) ulast = v;
            }
            if (yo >= 0 && yo < N) {
                const bool odd = cs[2 * NS - 1] & 1;
                *reinterpret_cast<float2*>(gu + static_cast<size_t>(yo) * N + 2 * tp) =
                    odd ? make_float2(uo_other, ulast) : make_float2(ulast, uo_other);
            }
            if (PRE && yr >= 0 && yr < N) {
                // restricted residual (same arithmetic as resid_restrict_cell)
                float sres = (yr & 1) ? racc : 0.0f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float up = ru[h];
                    float a2 = rkw[h] * (up - rw[h]);
                    a2 += rke[h] * (up - re[h]);
                    a2 += rkn[h] * (up - rn_[h]);
                    a2 += rks[h] * (up - rs[h]);
                    sres += rb[h] - ih2 * a2;
                }
                if (yr & 1) gbc[(yr >> 1) * Gm::NC + tp] = 0.25f * sres;
                else racc = sres;
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if (tp == 0 && act && !live) {
        // a wait gave up: let the bulk copies still in flight land before the CTA leaves
        const uint64_t t0 = now_ns();
        for (int s = 0; s < kRing && s < N; ++s) {
            const int r = s + ((N - 1 - s) / kRing) * kRing;  // last bundle of slot s
            while (!mbar_test(&full[s], (r / kRing) & 1) && now_ns() - t0 < 1000000000ull) {
            }
        }
    }
}

template <int N, int NS, bool PRE, bool POST>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_stream<N, NS, PRE, POST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(Geom<N>::bytes)) == cudaSuccess;
}

template <int N, int NS>
bool attrs_ns()
{
    return attr<N, NS, false, false>() && attr<N, NS, true, false>() && attr<N, NS, false, true>();
}

template <int N>
bool attrs_n()
{
    return attrs_ns<N, 1>() && attrs_ns<N, 2>();
}

template <int N, int NS>
void go(const FmgArgs& A, int t, int B, int ones, int first, bool pre, bool post, cudaStream_t st)
{
    using Gm = Geom<N>;
    const int grid = (B + Gm::G - 1) / Gm::G;
    if (pre) kb_rbgs_stream<N, NS, true, false><<<grid, kThreads, Gm::bytes, st>>>(A, t, B, ones, first);
    else if (post) kb_rbgs_stream<N, NS, false, true><<<grid, kThreads, Gm::bytes, st>>>(A, t, B, ones, first);
    else kb_rbgs_stream<N, NS, false, false><<<grid, kThreads, Gm::bytes, st>>>(A, t, B, ones, first);
}

template <int N>
void go_n(const FmgArgs& A, int t, int B, int ns, int ones, int first, bool pre, bool post, cudaStream_t st)
{
    if (ns == 2) go<N, 2>(A, t, B, ones, first, pre, post, st);
    else go<N, 1>(A, t, B, ones, first, pre, post, st);
}

}  // namespace

namespace mlqmc_stream {

bool supported(int n)
{
    return n == 8 || n == 16 || n == 32 || n == 64 || n == 128 || n == 256;
}

bool prepare()
{
    return attrs_n<8>() && attrs_n<16>() && attrs_n<32>() && attrs_n<64>() && attrs_n<128>() && attrs_n<256>();
}

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool pre, bool post, cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n || (ns != 1 && ns != 2) || (pre && post)) return false;
    switch (n) {
    case 8: go_n<8>(A, t, B, ns, ones, first, pre, post, st); break;
    case 16: go_n<16>(A, t, B, ns, ones, first, pre, post, st); break;
    case 32: go_n<32>(A, t, B, ns, ones, first, pre, post, st); break;
    case 64: go_n<64>(A, t, B, ns, ones, first, pre, post, st); break;
    case 128: go_n<128>(A, t, B, ns, ones, first, pre, post, st); break;
    default: go_n<256>(A, t, B, ns, ones, first, pre, post, st); break;
    }
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mlqmc_stream
