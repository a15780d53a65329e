// CUDA path of the MG-MLQMC library (sm_103a).
//
// Kernels:
//  k_points     shifted rank-1 lattice sequence / Philox MC bits -> normals (Sec. 3.2)
//  k_fmg<T,MX>  persistent per-sample solver: one CTA takes one sample from a
//               queue (largest level first), synthesises the KL field on every
//               level of its hierarchy (eq. truncatedKL), runs Full Multigrid
//               with red-black Gauss-Seidel V-cycles (Sec. 4, Fig. FMG) and
//               writes F_t and dF_t for every level t of that FMG (the recycled
//               solutions of eq. Upsilon-reuse). MX: FP32 V-cycles inside FP64
//               residual refinement.
//  k_sums       deterministic per (level, shift) reuse sums (eq. Upsilon-reuse).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "mlqmc_internal.h"

namespace {

constexpr int kStatusNotConverged = 1;
constexpr int kStatusCheck = 2;

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

__global__ void k_points(const SampleDesc* __restrict__ smp, int count, int s, int sampler, uint64_t seed,
                         const uint32_t* __restrict__ z, double* __restrict__ Y, uint64_t* __restrict__ bits)
{
    const int64_t total = static_cast<int64_t>(count) * s;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(idx / s);
        const int j = static_cast<int>(idx - static_cast<int64_t>(q) * s);
        const SampleDesc d = smp[q];
        const uint64_t x = point_bits(sampler, seed, z, d.level, d.r, d.n, j);
        const size_t o = static_cast<size_t>(d.canon) * s + j;
        if (bits) bits[o] = x;
        if (Y) {
            const double u = (static_cast<double>(x >> 11) + 0.5) * 0x1.0p-53;  // open (0,1)
            Y[o] = normcdfinv(u);
        }
    }
}

// ---------------------------------------------------------------------------
// Block-wide helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) t += red[w];  // fixed order: deterministic
        red[32] = t;
    }
    __syncthreads();
    const double t = red[32];
    __syncthreads();
    return t;
}

template <typename T>
struct Lv {
    int n;
    T* u;      // iterate (FMG solution on the current top level, correction below it)
    T* bc;     // right-hand side of the coarse correction equation
    T* kx;     // faces x: row i2, face f between cells f-1 and f, [i2*(n+1) + f]; f=0,n: 2k (boundary)
    T* ky;     // faces y: face g between rows g-1 and g, [g*n + i1]; g=0,n: 2k (boundary)
    T* idiag;  // 1 / (sum of the four face coefficients)
    T* k;      // coefficient exp(z) at cell centres
    T* G;      // KL partial sums, Ka x n
    double* u64;   // mixed forms: FP64 solution
    double* kx64;  // mixed forms: faces from the FP32 field, widened, in FP64
    double* ky64;
};

struct FmgArgs {
    const SampleDesc* samples;
    int n_samples;
    const double* Y;
    int s;
    int n0;
    int n_levels;
    int qoi;
    int mu0, nu1, nu2;
    double rtol;
    int max_iter;
    int Ka;
    const void* psi;
    size_t psi_off[MLQMC_MAX_LEVELS];
    const int* grp_start;
    const int* grp_b;
    const int* grp_m;
    const double* grp_sqrt;
    unsigned char* work;
    size_t slot_bytes;
    LevelOffsets lv[MLQMC_MAX_LEVELS];
    double* dF;
    double* F_out;
    double* usol;        // single-sample solution output (concatenated levels) or null
    double* k_out;       // field-only mode: k of level `field_level` per sample, or null
    int field_level;
    int* queue;
    int* status;
};

template <typename T>
__device__ __forceinline__ Lv<T> level_view(const FmgArgs& A, unsigned char* slot, int t)
{
    const LevelOffsets& o = A.lv[t];
    Lv<T> L;
    L.n = o.n;
    L.u = reinterpret_cast<T*>(slot + o.u);
    L.bc = reinterpret_cast<T*>(slot + o.bc);
    L.kx = reinterpret_cast<T*>(slot + o.kx);
    L.ky = reinterpret_cast<T*>(slot + o.ky);
    L.idiag = reinterpret_cast<T*>(slot + o.idiag);
    L.k = reinterpret_cast<T*>(slot + o.k);
    L.G = reinterpret_cast<T*>(slot + o.G);
    L.u64 = reinterpret_cast<double*>(slot + o.u64);
    L.kx64 = reinterpret_cast<double*>(slot + o.kx64);
    L.ky64 = reinterpret_cast<double*>(slot + o.ky64);
    return L;
}

__device__ __forceinline__ float expT(float x) { return expf(x); }
__device__ __forceinline__ double expT(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T hmean(T a, T b)
{
    return T(2) * a * b / (a + b);
}

// KL field on one level (eq. truncatedKL at the level's own cell centres):
// z(x1,x2) = sum_a psi_a(x1) G_a(x2), G_a(x2) = sum_{m: a_m = a} sqrt(theta_m) y_m psi_{b_m}(x2);
// then k = exp(z), harmonic-mean faces and the inverse diagonal.
template <typename T, bool MX>
__device__ void synth_level(const FmgArgs& A, const Lv<T>& L, int t, const double* cy)
{
    const int n = L.n;
    const T* psi = static_cast<const T*>(A.psi) + A.psi_off[t];
    const int Ka = A.Ka;
    for (int idx = threadIdx.x; idx < Ka * n; idx += blockDim.x) {
        const int a = idx / n;
        const int i2 = idx - a * n;
        T acc = T(0);
        const int g1 = A.grp_start[a + 1];
        for (int g = A.grp_start[a]; g < g1; ++g) acc += static_cast<T>(cy[g]) * psi[A.grp_b[g] * n + i2];
        L.G[idx] = acc;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n;
        const int i1 = p - i2 * n;
        T z = T(0);
        for (int a = 0; a < Ka; ++a) z += psi[a * n + i1] * L.G[a * n + i2];
        L.k[p] = expT(z);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * (n + 1); idx += blockDim.x) {
        const int i2 = idx / (n + 1);
        const int f = idx - i2 * (n + 1);
        const T* kr = L.k + i2 * n;
        T v;
        if (f == 0) v = T(2) * kr[0];
        else if (f == n) v = T(2) * kr[n - 1];
        else v = hmean(kr[f - 1], kr[f]);
        L.kx[idx] = v;
        // y faces: face g = idx / n between rows g-1 and g
        const int g = idx / n;
        const int i1 = idx - g * n;
        T w;
        if (g == 0) w = T(2) * L.k[i1];
        else if (g == n) w = T(2) * L.k[(n - 1) * n + i1];
        else w = hmean(L.k[(g - 1) * n + i1], L.k[g * n + i1]);
        L.ky[idx] = w;
        if constexpr (MX) {
            double v64, w64;
            if (f == 0) v64 = 2.0 * static_cast<double>(kr[0]);
            else if (f == n) v64 = 2.0 * static_cast<double>(kr[n - 1]);
            else v64 = hmean(static_cast<double>(kr[f - 1]), static_cast<double>(kr[f]));
            if (g == 0) w64 = 2.0 * static_cast<double>(L.k[i1]);
            else if (g == n) w64 = 2.0 * static_cast<double>(L.k[(n - 1) * n + i1]);
            else w64 = hmean(static_cast<double>(L.k[(g - 1) * n + i1]), static_cast<double>(L.k[g * n + i1]));
            L.kx64[idx] = v64;
            L.ky64[idx] = w64;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n;
        const int i1 = p - i2 * n;
        const T d = L.kx[i2 * (n + 1) + i1] + L.kx[i2 * (n + 1) + i1 + 1] + L.ky[i2 * n + i1] + L.ky[(i2 + 1) * n + i1];
        L.idiag[p] = T(1) / d;
    }
    __syncthreads();
}

// One red-black Gauss-Seidel half sweep (colour 0: i1+i2 even). b == null: b = 1.
template <typename T>
__device__ __forceinline__ void gs_colour(const Lv<T>& L, const T* b, int colour)
{
    const int n = L.n;
    const int half = n >> 1;
    const T h2 = T(1) / (T(n) * T(n));
    for (int idx = threadIdx.x; idx < n * half; idx += blockDim.x) {
        const int i2 = idx / half;
        const int i1 = 2 * (idx - i2 * half) + ((i2 + colour) & 1);
        const int p = i2 * n + i1;
        const T* kx = L.kx + i2 * (n + 1);
        T acc = h2 * (b ? b[p] : T(1));
        if (i1 > 0) acc += kx[i1] * L.u[p - 1];
        if (i1 < n - 1) acc += kx[i1 + 1] * L.u[p + 1];
        if (i2 > 0) acc += L.ky[i2 * n + i1] * L.u[p - n];
        if (i2 < n - 1) acc += L.ky[(i2 + 1) * n + i1] * L.u[p + n];
        L.u[p] = acc * L.idiag[p];
    }
    __syncthreads();
}

// (A u)_P scaled by h^2 in flux form: sum over faces k_f (u_P - u_Q), with
// u_Q = 0 across the boundary (where k_f holds 2 k_P). Differences of
// neighbouring values keep the FP64 residual floor near eps * |flux|.
template <typename T, typename U>
__device__ __forceinline__ U apply_h2(const T* kx, const T* ky, const U* u, int n, int i1, int i2)
{
    const int p = i2 * n + i1;
    const U up = u[p];
    U acc = U(kx[i2 * (n + 1) + i1]) * (up - (i1 > 0 ? u[p - 1] : U(0)));
    acc += U(kx[i2 * (n + 1) + i1 + 1]) * (up - (i1 < n - 1 ? u[p + 1] : U(0)));
    acc += U(ky[i2 * n + i1]) * (up - (i2 > 0 ? u[p - n] : U(0)));
    acc += U(ky[(i2 + 1) * n + i1]) * (up - (i2 < n - 1 ? u[p + n] : U(0)));
    return acc;
}

// r = b - A u on the fine level, restricted by the mean of the four children.
template <typename T>
__device__ void resid_restrict(const Lv<T>& F, const T* b, T* bc)
{
    const int n = F.n;
    const int nc = n >> 1;
    const T ih2 = T(n) * T(n);
    for (int idx = threadIdx.x; idx < nc * nc; idx += blockDim.x) {
        const int I2 = idx / nc;
        const int I1 = idx - I2 * nc;
        T s = T(0);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int i1 = 2 * I1 + (d & 1), i2 = 2 * I2 + (d >> 1);
            const int p = i2 * n + i1;
            s += (b ? b[p] : T(1)) - ih2 * apply_h2<T, T>(F.kx, F.ky, F.u, n, i1, i2);
        }
        bc[idx] = T(0.25) * s;
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T ghost(const T* e, int nc, int I1, int I2)
{
    T sg = T(1);
    if (I1 < 0) { I1 = 0; sg = -sg; }
    if (I1 >= nc) { I1 = nc - 1; sg = -sg; }
    if (I2 < 0) { I2 = 0; sg = -sg; }
    if (I2 >= nc) { I2 = nc - 1; sg = -sg; }
    return sg * e[I2 * nc + I1];
}

// Bilinear cell-centred prolongation (9,3,3,1)/16 with odd reflection at the
// Dirichlet boundary; ADD: fine += P e, else fine = P e.
template <typename S, typename D, bool ADD>
__device__ void prolong(const S* e, int nc, D* fine)
{
    const int nf = 2 * nc;
    for (int p = threadIdx.x; p < nf * nf; p += blockDim.x) {
        const int i2 = p / nf;
        const int i1 = p - i2 * nf;
        const int I1 = i1 >> 1, I2 = i2 >> 1;
        const int s1 = (i1 & 1) ? 1 : -1, s2 = (i2 & 1) ? 1 : -1;
        const D v = D(9) * D(ghost(e, nc, I1, I2)) + D(3) * D(ghost(e, nc, I1 + s1, I2)) +
                    D(3) * D(ghost(e, nc, I1, I2 + s2)) + D(ghost(e, nc, I1 + s1, I2 + s2));
        if (ADD) fine[p] += v * D(0.0625);
        else fine[p] = v * D(0.0625);
    }
    __syncthreads();
}

// Banded Cholesky of h0^2 A_0 (bandwidth n0), warp 0. Lb[i*(n0+1) + d] = L(i, i-d).
template <typename F>
__device__ void chol_factor(double* Lb, int n0, const F* kx, const F* ky)
{
    if (threadIdx.x < 32) {
        const int N = n0 * n0, W = n0 + 1, lane = threadIdx.x;
        for (int j = 0; j < N; ++j) {
            const int j1 = j % n0, j2 = j / n0;
            double d = static_cast<double>(kx[j2 * (n0 + 1) + j1]) + static_cast<double>(kx[j2 * (n0 + 1) + j1 + 1]) +
                       static_cast<double>(ky[j2 * n0 + j1]) + static_cast<double>(ky[(j2 + 1) * n0 + j1]);
            for (int q = 1; q <= n0 && q <= j; ++q) {
                const double l = Lb[j * W + q];
                d -= l * l;
            }
            const double Ljj = sqrt(d);
            if (lane == 0) Lb[j * W] = Ljj;
            if (lane >= 1 && lane <= n0 && j + lane < N) {
                const int i = j + lane;
                const int i1 = i % n0, i2 = i / n0;
                double a = 0.0;
                if (lane == 1 && i1 > 0) a = -static_cast<double>(kx[i2 * (n0 + 1) + i1]);
                if (lane == n0) a = -static_cast<double>(ky[i2 * n0 + i1]);
                for (int tt = (i - n0 > 0 ? i - n0 : 0); tt < j; ++tt) a -= Lb[i * W + (i - tt)] * Lb[j * W + (j - tt)];
                Lb[i * W + lane] = a / Ljj;
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

// Solve (h0^2 A_0) x = h0^2 b with the band factor; b == null: b = 1. Thread 0.
template <typename B, typename X>
__device__ void chol_solve(const double* Lb, int n0, const B* b, X* x, double* tmp)
{
    if (threadIdx.x == 0) {
        const int N = n0 * n0, W = n0 + 1;
        const double h2 = 1.0 / (static_cast<double>(n0) * n0);
        for (int i = 0; i < N; ++i) {
            double v = h2 * (b ? static_cast<double>(b[i]) : 1.0);
            for (int q = 1; q <= n0 && q <= i; ++q) v -= Lb[i * W + q] * tmp[i - q];
            tmp[i] = v / Lb[i * W];
        }
        for (int i = N - 1; i >= 0; --i) {
            double v = tmp[i];
            for (int q = 1; q <= n0 && i + q < N; ++q) v -= Lb[(i + q) * W + q] * tmp[i + q];
            tmp[i] = v / Lb[i * W];
        }
        for (int i = 0; i < N; ++i) x[i] = static_cast<X>(tmp[i]);
    }
    __syncthreads();
}

template <typename T>
__device__ void zero(T* a, int cnt)
{
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) a[p] = T(0);
    __syncthreads();
}

// V-cycle (Sec. 4 correction scheme, recursively) on levels t_top..0.
// top_b == null: right-hand side 1 on the top level.
template <typename T>
__device__ void vcycle(const FmgArgs& A, unsigned char* slot, int t_top, const T* top_b, const double* Lb, double* tmp)
{
    for (int t = t_top; t >= 1; --t) {
        const Lv<T> F = level_view<T>(A, slot, t);
        const T* b = (t == t_top) ? top_b : F.bc;
        if (t < t_top) zero(F.u, F.n * F.n);
        for (int s = 0; s < A.nu1; ++s) {
            gs_colour(F, b, 0);
            gs_colour(F, b, 1);
        }
        const Lv<T> Cl = level_view<T>(A, slot, t - 1);
        resid_restrict(F, b, Cl.bc);
    }
    {
        const Lv<T> C0 = level_view<T>(A, slot, 0);
        chol_solve(Lb, A.n0, t_top == 0 ? top_b : C0.bc, C0.u, tmp);
    }
    for (int t = 1; t <= t_top; ++t) {
        const Lv<T> F = level_view<T>(A, slot, t);
        const Lv<T> Cl = level_view<T>(A, slot, t - 1);
        prolong<T, T, true>(Cl.u, Cl.n, F.u);
        const T* b = (t == t_top) ? top_b : F.bc;
        for (int s = 0; s < A.nu2; ++s) {
            gs_colour(F, b, 1);
            gs_colour(F, b, 0);
        }
    }
}

// ||1 - A u||_2 on one level (b = 1), FP64 accumulation.
template <typename T>
__device__ double resid_norm_ones(const Lv<T>& L, double* red)
{
    const int n = L.n;
    const double ih2 = static_cast<double>(n) * n;
    double acc = 0.0;
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n, i1 = p - i2 * n;
        const double r = 1.0 - ih2 * static_cast<double>(apply_h2<T, T>(L.kx, L.ky, L.u, n, i1, i2));
        acc += r * r;
    }
    return sqrt(block_sum(acc, red));
}

// Mixed forms: r = 1 - A64 u64 in FP64, stored to the FP32 rhs; returns ||r||_2.
__device__ double resid64_to_rhs(const Lv<float>& L, double* red)
{
    const int n = L.n;
    const double ih2 = static_cast<double>(n) * n;
    double acc = 0.0;
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n, i1 = p - i2 * n;
        const double r = 1.0 - ih2 * apply_h2<double, double>(L.kx64, L.ky64, L.u64, n, i1, i2);
        L.bc[p] = static_cast<float>(r);
        acc += r * r;
    }
    return sqrt(block_sum(acc, red));
}

template <typename T>
__device__ double qoi(const T* u, int n, int kind, double* red)
{
    if (kind == MLQMC_QOI_MEAN) {
        double acc = 0.0;
        for (int p = threadIdx.x; p < n * n; p += blockDim.x) acc += static_cast<double>(u[p]);
        return block_sum(acc, red) / (static_cast<double>(n) * n);
    }
    const int m = n / 2;
    const double v = 0.25 * (static_cast<double>(u[(m - 1) * n + (m - 1)]) + static_cast<double>(u[(m - 1) * n + m]) +
                             static_cast<double>(u[m * n + (m - 1)]) + static_cast<double>(u[m * n + m]));
    __syncthreads();
    return v;
}

template <typename T>
__device__ void copy_out(const T* src, double* dst, int cnt)
{
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) dst[p] = static_cast<double>(src[p]);
    __syncthreads();
}

// Persistent FMG kernel. Shared memory: cy[s] | Lb[n0^2 (n0+1)] | tmp[n0^2] | red[40] | F[16].
template <typename T, bool MX>
__global__ void __launch_bounds__(256) k_fmg(FmgArgs A)
{
    extern __shared__ double smem[];
    double* cy = smem;
    const int N0 = A.n0 * A.n0;
    double* Lb = cy + ((A.s + 1) & ~1);
    double* tmp = Lb + N0 * (A.n0 + 1);
    double* red = tmp + N0;
    double* Fv = red + 40;
    __shared__ int s_q;
    unsigned char* slot = A.work + static_cast<size_t>(blockIdx.x) * A.slot_bytes;

    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(A.queue, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= A.n_samples) break;
        const SampleDesc d = A.samples[q];
        const int Lf = d.level;
        // sqrt(theta_m) y_m in grouped-by-a order
        for (int g = threadIdx.x; g < A.s; g += blockDim.x)
            cy[g] = A.grp_sqrt[g] * A.Y[static_cast<size_t>(d.canon) * A.s + A.grp_m[g]];
        __syncthreads();

        if (A.k_out) {  // field-only mode (introspection)
            const Lv<T> L = level_view<T>(A, slot, A.field_level);
            synth_level<T, MX>(A, L, A.field_level, cy);
            copy_out(L.k, A.k_out + static_cast<size_t>(d.canon) * L.n * L.n, L.n * L.n);
            continue;
        }

        for (int t = 0; t <= Lf; ++t) synth_level<T, MX>(A, level_view<T>(A, slot, t), t, cy);

        size_t uoff = 0;
        {
            const Lv<T> L0 = level_view<T>(A, slot, 0);
            if constexpr (MX) {
                chol_factor(Lb, A.n0, L0.kx64, L0.ky64);
                chol_solve<T, double>(Lb, A.n0, nullptr, L0.u64, tmp);
                const double F0 = qoi(L0.u64, A.n0, A.qoi, red);
                if (threadIdx.x == 0) Fv[0] = F0;
                if (A.usol) copy_out(L0.u64, A.usol, N0);
            } else {
                chol_factor(Lb, A.n0, L0.kx, L0.ky);
                chol_solve<T, T>(Lb, A.n0, nullptr, L0.u, tmp);
                const double F0 = qoi(L0.u, A.n0, A.qoi, red);
                if (threadIdx.x == 0) Fv[0] = F0;
                if (A.usol) copy_out(L0.u, A.usol, N0);
            }
            uoff = N0;
        }
        for (int t = 1; t <= Lf; ++t) {
            const Lv<T> L = level_view<T>(A, slot, t);
            const Lv<T> Lc = level_view<T>(A, slot, t - 1);
            const int n = L.n;
            double Ft;
            if constexpr (MX) {
                prolong<double, double, false>(Lc.u64, Lc.n, L.u64);
                for (int m = 0; m < A.mu0; ++m) {
                    // one refinement step per FMG cycle: r = 1 - A64 u64, FP32 V-cycle on A e = r
                    resid64_to_rhs(L, red);
                    zero(L.u, n * n);
                    vcycle<T>(A, slot, t, L.bc, Lb, tmp);
                    for (int p = threadIdx.x; p < n * n; p += blockDim.x) L.u64[p] += static_cast<double>(L.u[p]);
                    __syncthreads();
                }
                if (A.rtol > 0.0) {
                    int it = 0;
                    for (;;) {
                        const double rn = resid64_to_rhs(L, red);
                        if (rn <= A.rtol * n) break;
                        if (it >= A.max_iter) {
                            if (threadIdx.x == 0) atomicOr(A.status, kStatusNotConverged);
                            break;
                        }
                        zero(L.u, n * n);
                        vcycle<T>(A, slot, t, L.bc, Lb, tmp);
                        for (int p = threadIdx.x; p < n * n; p += blockDim.x) L.u64[p] += static_cast<double>(L.u[p]);
                        __syncthreads();
                        ++it;
                    }
                }
                Ft = qoi(L.u64, n, A.qoi, red);
                if (A.usol) copy_out(L.u64, A.usol + uoff, n * n);
            } else {
                prolong<T, T, false>(Lc.u, Lc.n, L.u);
                for (int m = 0; m < A.mu0; ++m) vcycle<T>(A, slot, t, nullptr, Lb, tmp);
                if (A.rtol > 0.0) {
                    int it = 0;
                    for (;;) {
                        const double rn = resid_norm_ones(L, red);
                        if (rn <= A.rtol * n) break;
                        if (it >= A.max_iter) {
                            if (threadIdx.x == 0) atomicOr(A.status, kStatusNotConverged);
                            break;
                        }
                        vcycle<T>(A, slot, t, nullptr, Lb, tmp);
                        ++it;
                    }
                }
                Ft = qoi(L.u, n, A.qoi, red);
                if (A.usol) copy_out(L.u, A.usol + uoff, n * n);
            }
            if (threadIdx.x == 0) Fv[t] = Ft;
            uoff += static_cast<size_t>(n) * n;
        }
        __syncthreads();
        if (threadIdx.x < A.n_levels) {
            const int t = threadIdx.x;
            const size_t o = static_cast<size_t>(d.canon) * A.n_levels + t;
            const double Ft = t <= Lf ? Fv[t] : 0.0;
            const double dF = t <= Lf ? Ft - (t > 0 ? Fv[t - 1] : 0.0) : 0.0;
            if (A.dF) A.dF[o] = dF;
            if (A.F_out) A.F_out[o] = Ft;
        }
        __syncthreads();
    }
}

// Deterministic reuse sums per (level t, shift r): one block each, fixed order.
__global__ void k_sums(const int2* __restrict__ canon, int n, const double* __restrict__ dF, int n_levels, int R,
                       int reuse, double* __restrict__ sums)
{
    __shared__ double red[48];
    const int t = blockIdx.x / R;
    const int r = blockIdx.x - t * R;
    double a = 0.0, a2 = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int2 lr = canon[q];
        if (lr.y == r && (reuse ? lr.x >= t : lr.x == t)) {
            const double v = dF[static_cast<size_t>(q) * n_levels + t];
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

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
inline bool ok(cudaError_t e) { return e == cudaSuccess; }

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool is_mixed(const mlqmc_problem& p) { return p.precision != MLQMC_FP64; }

SlotLayout make_layout(const mlqmc_problem& p, int Ka)
{
    SlotLayout L;
    L.n_levels = p.n_levels;
    const size_t es = is_mixed(p) ? sizeof(float) : sizeof(double);
    size_t off = 0;
    for (int t = 0; t < p.n_levels; ++t) {
        const size_t n = static_cast<size_t>(p.coarse_cells) << t;
        LevelOffsets& o = L.lv[t];
        o.n = static_cast<int>(n);
        o.u = off; off = align256(off + es * n * n);
        o.bc = off; off = align256(off + es * n * n);
        o.kx = off; off = align256(off + es * n * (n + 1));
        o.ky = off; off = align256(off + es * n * (n + 1));
        o.idiag = off; off = align256(off + es * n * n);
        o.k = off; off = align256(off + es * n * n);
        o.G = off; off = align256(off + es * Ka * n);
        if (is_mixed(p)) {
            o.u64 = off; off = align256(off + 8 * n * n);
            o.kx64 = off; off = align256(off + 8 * n * (n + 1));
            o.ky64 = off; off = align256(off + 8 * n * (n + 1));
        } else {
            o.u64 = o.kx64 = o.ky64 = 0;
        }
    }
    L.bytes = off;
    return L;
}

size_t fmg_smem_bytes(const mlqmc_problem& p)
{
    const size_t N0 = static_cast<size_t>(p.coarse_cells) * p.coarse_cells;
    return sizeof(double) * (((p.n_modes + 1) & ~1) + N0 * (p.coarse_cells + 1) + N0 + 40 + 16);
}

template <typename T, bool MX>
void* fmg_kernel_ptr()
{
    return reinterpret_cast<void*>(&k_fmg<T, MX>);
}

void* fmg_kernel(const mlqmc_problem& p)
{
    return is_mixed(p) ? fmg_kernel_ptr<float, true>() : fmg_kernel_ptr<double, false>();
}

FmgArgs base_args(mlqmc_ctx* c)
{
    FmgArgs A;
    std::memset(&A, 0, sizeof(A));
    A.Y = c->d_Y;
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
    A.work = c->d_work;
    A.slot_bytes = c->layout.bytes;
    for (int t = 0; t < c->p.n_levels; ++t) A.lv[t] = c->layout.lv[t];
    A.queue = c->d_queue;
    A.status = c->d_status;
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

// Record the opening event of a timed launch (no-op unless profiling).
cudaEvent_t mark_begin(mlqmc_ctx* c, cudaStream_t st)
{
    if (!c->profiling) return nullptr;
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, st);
    return e;
}

void mark_end(mlqmc_ctx* c, int kind, cudaEvent_t a, cudaStream_t st)
{
    if (!a) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, st);
    c->marks.push_back({kind, a, b});
}

mlqmc_status launch_fmg(mlqmc_ctx* c, FmgArgs& A, int n_samples, cudaStream_t st)
{
    A.n_samples = n_samples;
    if (!ok(cudaMemsetAsync(c->d_queue, 0, sizeof(int), st))) return MLQMC_ERR_CUDA;
    const int grid = std::max(1, std::min(n_samples, c->slots));
    void* args[] = {&A};
    cudaEvent_t m = mark_begin(c, st);
    if (!ok(cudaLaunchKernel(fmg_kernel(c->p), dim3(grid), dim3(c->fmg_threads), args, c->fmg_smem, st)))
        return MLQMC_ERR_CUDA;
    mark_end(c, 1, m, st);
    c->launches += 1;
    return MLQMC_OK;
}

mlqmc_status launch_points(mlqmc_ctx* c, const SampleDesc* d_s, int count, double* Y, uint64_t* bits, cudaStream_t st)
{
    const int64_t total = static_cast<int64_t>(count) * c->p.n_modes;
    const int threads = 256;
    const int64_t want = (total + threads - 1) / threads;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(c->sm_count) * 16)));
    cudaEvent_t m = mark_begin(c, st);
    k_points<<<grid, threads, 0, st>>>(d_s, count, c->p.n_modes, c->p.sampler, c->p.seed, c->d_z, Y, bits);
    if (!ok(cudaGetLastError())) return MLQMC_ERR_CUDA;
    mark_end(c, 0, m, st);
    c->launches += 1;
    return MLQMC_OK;
}

void free_ctx(mlqmc_ctx* c)
{
    if (!c) return;
    cudaFree(c->d_psi);
    cudaFree(c->d_psi32);
    cudaFree(c->d_grp_start);
    cudaFree(c->d_grp_b);
    cudaFree(c->d_grp_m);
    cudaFree(c->d_grp_sqrt);
    cudaFree(c->d_z);
    cudaFree(c->d_samples);
    cudaFree(c->d_canon);
    cudaFree(c->d_Y);
    cudaFree(c->d_dF);
    cudaFree(c->d_work);
    cudaFree(c->d_status);
    cudaFree(c->d_queue);
    if (c->staged) cudaEventDestroy(c->staged);
    for (auto& m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->h_samples) cudaFreeHost(c->h_samples);
    if (c->h_canon) cudaFreeHost(c->h_canon);
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
    if (p->sampler == MLQMC_SAMPLER_LATTICE) {
        if (!p->genvec || p->log2_nmax < 0 || p->log2_nmax > 32) return MLQMC_ERR_INVALID_ARG;
        for (int j = 0; j < p->n_modes; ++j)
            if ((p->genvec[j] & 1u) == 0) return MLQMC_ERR_INVALID_ARG;
    }
    return MLQMC_OK;
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

    // KL tables (Sec. 5): modes, 1D eigenpairs, per-level psi tables
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
    std::vector<float> psi32;
    size_t off = 0;
    for (int t = 0; t < p->n_levels; ++t) {
        const int n = p->coarse_cells << t;
        mlqmc::psi_table(c->eig, p->corr_len, K1, n, tab);
        c->psi_off[t] = off;
        psi_all.insert(psi_all.end(), tab.begin(), tab.end());
        off += tab.size();
    }
    psi32.assign(psi_all.begin(), psi_all.end());
    bool good = dev_upload(&c->d_psi, psi_all.data(), psi_all.size()) &&
                dev_upload(&c->d_psi32, psi32.data(), psi32.size()) &&
                dev_upload(&c->d_grp_start, gstart.data(), gstart.size()) &&
                dev_upload(&c->d_grp_b, gb.data(), gb.size()) && dev_upload(&c->d_grp_m, gm.data(), gm.size()) &&
                dev_upload(&c->d_grp_sqrt, gsq.data(), gsq.size()) &&
                dev_upload(&c->d_z, c->z.data(), c->z.size());
    if (!good) {
        free_ctx(c);
        return MLQMC_ERR_OOM;
    }

    // per-call buffers
    c->max_samples = max_samples_per_call > 0 ? max_samples_per_call : 65536;
    const size_t ms = static_cast<size_t>(c->max_samples);
    good = ok(cudaMalloc(&c->d_samples, ms * sizeof(SampleDesc))) && ok(cudaMalloc(&c->d_canon, ms * sizeof(int2))) &&
           ok(cudaMalloc(&c->d_Y, ms * p->n_modes * sizeof(double))) &&
           ok(cudaMalloc(&c->d_dF, (ms + 1) * p->n_levels * sizeof(double))) &&
           ok(cudaMallocHost(&c->h_samples, ms * sizeof(SampleDesc))) &&
           ok(cudaMallocHost(&c->h_canon, ms * sizeof(int2))) && ok(cudaMalloc(&c->d_status, sizeof(int))) &&
           ok(cudaMalloc(&c->d_queue, sizeof(int))) && ok(cudaMemset(c->d_status, 0, sizeof(int))) &&
           ok(cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming));
    if (!good) {
        free_ctx(c);
        return MLQMC_ERR_OOM;
    }

    // FMG workspace: one slot per resident CTA, capped by a memory budget
    c->layout = make_layout(c->p, Ka);
    c->fmg_smem = fmg_smem_bytes(c->p);
    void* kern = fmg_kernel(c->p);
    if (c->fmg_smem > 48 * 1024 &&
        !ok(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(c->fmg_smem)))) {
        free_ctx(c);
        return MLQMC_ERR_CUDA;
    }
    int per_sm = 0;
    if (!ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c->fmg_threads, c->fmg_smem)) || per_sm < 1) {
        free_ctx(c);
        return MLQMC_ERR_CUDA;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t budget = std::min<size_t>(free_b / 2, static_cast<size_t>(48) << 30);
    int64_t slots = static_cast<int64_t>(c->sm_count) * per_sm;
    slots = std::min<int64_t>(slots, static_cast<int64_t>(budget / std::max<size_t>(1, c->layout.bytes)));
    slots = std::min<int64_t>(slots, c->max_samples);
    if (slots < 1) {
        free_ctx(c);
        return MLQMC_ERR_OOM;
    }
    c->slots = static_cast<int>(slots);
    if (!ok(cudaMalloc(&c->d_work, static_cast<size_t>(c->slots) * c->layout.bytes))) {
        free_ctx(c);
        return MLQMC_ERR_OOM;
    }
    *out = c;
    return MLQMC_OK;
}

extern "C" void mlqmc_destroy(mlqmc_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_ctx(c);
}

extern "C" mlqmc_status mlqmc_sample_levels(mlqmc_ctx* c, const mlqmc_work* work, int32_t n_work, double* d_sums,
                                            double* d_F, void* stream)
{
    if (!c || n_work < 0 || (n_work > 0 && !work) || !d_sums) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const mlqmc_problem& p = c->p;
    // validate and count
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
    // expand in work order, process in chunks of max_samples
    int item = 0, rr = n_work > 0 ? work[0].r_begin : 0;
    int64_t nn = n_work > 0 ? work[0].n_begin : 0;
    int64_t done = 0;
    while (done < total) {
        const int64_t chunk = std::min<int64_t>(total - done, c->max_samples);
        // the pinned staging buffers may still feed an earlier call's copies
        if (!ok(cudaEventSynchronize(c->staged))) return MLQMC_ERR_CUDA;
        std::vector<SampleDesc> buf;
        buf.reserve(chunk);
        for (int64_t q = 0; q < chunk; ++q) {
            while (item < n_work && (work[item].n_end == work[item].n_begin || work[item].r_end == work[item].r_begin ||
                                     rr >= work[item].r_end)) {
                ++item;
                if (item < n_work) {
                    rr = work[item].r_begin;
                    nn = work[item].n_begin;
                }
            }
            SampleDesc d;
            d.n = nn;
            d.r = rr;
            d.level = work[item].level;
            d.canon = static_cast<int32_t>(q);
            d.pad = 0;
            buf.push_back(d);
            c->h_canon[q] = make_int2(d.level, d.r);
            if (++nn >= work[item].n_end) {
                nn = work[item].n_begin;
                ++rr;
            }
        }
        // queue order: largest level first (stable), so long solves start early
        std::stable_sort(buf.begin(), buf.end(), [](const SampleDesc& x, const SampleDesc& y) { return x.level > y.level; });
        std::memcpy(c->h_samples, buf.data(), chunk * sizeof(SampleDesc));
        if (!ok(cudaMemcpyAsync(c->d_samples, c->h_samples, chunk * sizeof(SampleDesc), cudaMemcpyHostToDevice, st)) ||
            !ok(cudaMemcpyAsync(c->d_canon, c->h_canon, chunk * sizeof(int2), cudaMemcpyHostToDevice, st)) ||
            !ok(cudaEventRecord(c->staged, st)))
            return MLQMC_ERR_CUDA;
        mlqmc_status s1 = launch_points(c, c->d_samples, static_cast<int>(chunk), c->d_Y, nullptr, st);
        if (s1 != MLQMC_OK) return s1;
        FmgArgs A = base_args(c);
        A.samples = c->d_samples;
        A.dF = c->d_dF;
        A.F_out = d_F ? d_F + done * p.n_levels : nullptr;
        s1 = launch_fmg(c, A, static_cast<int>(chunk), st);
        if (s1 != MLQMC_OK) return s1;
        cudaEvent_t m = mark_begin(c, st);
        k_sums<<<p.n_levels * p.n_shifts, 256, 0, st>>>(c->d_canon, static_cast<int>(chunk), c->d_dF, p.n_levels,
                                                        p.n_shifts, p.reuse, d_sums);
        if (!ok(cudaGetLastError())) return MLQMC_ERR_CUDA;
        mark_end(c, 2, m, st);
        c->launches += 1;
        done += chunk;
    }
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
    if (h & kStatusNotConverged) return MLQMC_ERR_NOT_CONVERGED;
    if (h & kStatusCheck) return MLQMC_ERR_DEVICE_STATUS;
    return MLQMC_OK;
}

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
    if (!ok(cudaEventSynchronize(c->staged))) return MLQMC_ERR_CUDA;
    for (int i = 0; i < count; ++i) {
        SampleDesc d;
        d.n = n_begin + i;
        d.r = r;
        d.level = level;
        d.canon = i;
        d.pad = 0;
        c->h_samples[i] = d;
    }
    if (count > 0 &&
        (!ok(cudaMemcpyAsync(c->d_samples, c->h_samples, count * sizeof(SampleDesc), cudaMemcpyHostToDevice, st)) ||
         !ok(cudaEventRecord(c->staged, st))))
        return MLQMC_ERR_CUDA;
    return MLQMC_OK;
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
    if (!c || !d_y || !d_k || t < 0 || t >= c->p.n_levels || count < 0 || count > c->max_samples)
        return MLQMC_ERR_INVALID_ARG;
    if (count == 0) return MLQMC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, t, 0, 0, count, st, false);
    if (s != MLQMC_OK) return s;
    if (!ok(cudaMemcpyAsync(c->d_Y, d_y, static_cast<size_t>(count) * c->p.n_modes * sizeof(double),
                            cudaMemcpyDeviceToDevice, st)))
        return MLQMC_ERR_CUDA;
    FmgArgs A = base_args(c);
    A.samples = c->d_samples;
    A.k_out = d_k;
    A.field_level = t;
    return launch_fmg(c, A, count, st);
}

extern "C" mlqmc_status mlqmc_sample_solution(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n, double* d_u,
                                              double* d_F, void* stream)
{
    if (!c || !d_u || !d_F) return MLQMC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlqmc_status s = stage_block(c, level, r, n, 1, st);
    if (s != MLQMC_OK) return s;
    s = launch_points(c, c->d_samples, 1, c->d_Y, nullptr, st);
    if (s != MLQMC_OK) return s;
    FmgArgs A = base_args(c);
    A.samples = c->d_samples;
    A.dF = c->d_dF;
    A.usol = d_u;
    // F_0..F_level land in the first row of a scratch block, then copied out
    A.F_out = c->d_dF + c->p.n_levels;
    s = launch_fmg(c, A, 1, st);
    if (s != MLQMC_OK) return s;
    if (!ok(cudaMemcpyAsync(d_F, c->d_dF + c->p.n_levels, (level + 1) * sizeof(double), cudaMemcpyDeviceToDevice, st)))
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
    for (int i = 0; i < 3; ++i) {
        c->prof_ms[i] = 0.0;
        c->prof_n[i] = 0;
    }
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_profile_read(mlqmc_ctx* c, double* out_ms, int64_t* out_n)
{
    if (!c || !out_ms || !out_n) return MLQMC_ERR_INVALID_ARG;
    for (auto& m : c->marks) {
        if (!ok(cudaEventSynchronize(m.b))) return MLQMC_ERR_CUDA;
        float ms = 0.0f;
        if (!ok(cudaEventElapsedTime(&ms, m.a, m.b))) return MLQMC_ERR_CUDA;
        c->prof_ms[m.kind] += ms;
        c->prof_n[m.kind] += 1;
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    c->marks.clear();
    for (int i = 0; i < 3; ++i) {
        out_ms[i] = c->prof_ms[i];
        out_n[i] = c->prof_n[i];
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
        const int f = idx - i2 * (n + 1);
        const double* kr = L.k + i2 * n;
        L.kx[idx] = (f == 0) ? 2.0 * kr[0] : (f == n) ? 2.0 * kr[n - 1] : hmean(kr[f - 1], kr[f]);
        const int g = idx / n;
        const int i1 = idx - g * n;
        L.ky[idx] = (g == 0) ? 2.0 * L.k[i1]
                  : (g == n) ? 2.0 * L.k[(n - 1) * n + i1]
                             : hmean(L.k[(g - 1) * n + i1], L.k[g * n + i1]);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
        const int i2 = p / n;
        const int i1 = p - i2 * n;
        L.idiag[p] = 1.0 / (L.kx[i2 * (n + 1) + i1] + L.kx[i2 * (n + 1) + i1 + 1] + L.ky[i2 * n + i1] +
                            L.ky[(i2 + 1) * n + i1]);
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
    unsigned char* slot = A.work + static_cast<size_t>(blockIdx.x) * A.slot_bytes;
    const int Lf = A.n_levels - 1;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const double* ks = k_in + static_cast<size_t>(q) * k_stride;
        for (int t = 0; t <= Lf; ++t) {
            const Lv<double> L = level_view<double>(A, slot, t);
            for (int p = threadIdx.x; p < L.n * L.n; p += blockDim.x) L.k[p] = ks[p];
            ks += static_cast<size_t>(L.n) * L.n;
            __syncthreads();
            noalloc_faces(L);
        }
        const Lv<double> L0 = level_view<double>(A, slot, 0);
        chol_factor(Lb, A.n0, L0.kx, L0.ky);
        chol_solve<double, double>(Lb, A.n0, nullptr, L0.u, tmp);
        const double F0 = qoi(L0.u, A.n0, A.qoi, red);
        if (threadIdx.x == 0) Fv[0] = F0;
        for (int t = 1; t <= Lf; ++t) {
            const Lv<double> L = level_view<double>(A, slot, t);
            const Lv<double> Lc = level_view<double>(A, slot, t - 1);
            prolong<double, double, false>(Lc.u, Lc.n, L.u);
            for (int m = 0; m < A.mu0; ++m) vcycle<double>(A, slot, t, nullptr, Lb, tmp);
            const double Ft = qoi(L.u, L.n, A.qoi, red);
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
    if (coarse_cells > 16 || n_levels > 7 || (static_cast<int64_t>(coarse_cells) << (n_levels - 1)) > MLQMC_NOALLOC_MAX_CELLS)
        return MLQMC_ERR_SCRATCH_LIMIT;
    mlqmc_problem p{};
    p.n_levels = n_levels;
    p.coarse_cells = coarse_cells;
    p.n_modes = 1;
    p.precision = MLQMC_FP64;
    const SlotLayout lay = make_layout(p, 0);
    if (lay.bytes > static_cast<size_t>(MLQMC_NOALLOC_SLOT_BYTES)) return MLQMC_ERR_SCRATCH_LIMIT;
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
    A.work = scratch;
    A.slot_bytes = MLQMC_NOALLOC_SLOT_BYTES;
    for (int t = 0; t < n_levels; ++t) A.lv[t] = lay.lv[t];
    size_t k_stride = 0;
    for (int t = 0; t < n_levels; ++t) k_stride += static_cast<size_t>(lay.lv[t].n) * lay.lv[t].n;
    const size_t N0 = static_cast<size_t>(coarse_cells) * coarse_cells;
    const size_t smem = sizeof(double) * (N0 * (coarse_cells + 1) + N0 + 40 + 16);
    const int grid = std::min<int>(count, MLQMC_NOALLOC_SLOTS);
    k_fmg_noalloc<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(A, d_k, k_stride, count, d_F);
    return ok(cudaGetLastError()) ? MLQMC_OK : MLQMC_ERR_CUDA;
}

extern "C" int64_t mlqmc_launch_count(const mlqmc_ctx* c)
{
    return c ? c->launches : 0;
}
