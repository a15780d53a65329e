// Device-side building blocks of the FMG solver: per-sample level views over
// the level pools, the KL field, red-black Gauss-Seidel, residual/restriction,
// prolongation, the banded exact solve on level 0 and the V-cycle (Sec. 4).
// Every function here is called by all threads of a team (a CTA or one warp)
// working on one sample.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fastdiv.h"
#include "mlqmc_internal.h"

namespace mlqmc_dev {

constexpr int kStatusNotConverged = 1;
constexpr int kStatusCheck = 2;
constexpr int kStatusTimeout = 4;  // a bounded device wait gave up (tensor-core KL pipeline)

// Row pitch (elements) of the x-face array of an n x n level: n + 1 faces per
// row padded to n + 4, so that every row starts on a 16-byte boundary.
__host__ __device__ constexpr int kx_pitch(int n) { return n + 4; }

// Array of per-sample blocks: block i starts at base + i * stride (bytes).
struct ArrDesc {
    unsigned char* base;
    size_t stride;
};

struct LevelDesc {
    int n;
    ArrDesc u, bc, kx, ky, idiag, k, G, u64, u2;  // u2: ping-pong partner of u for the tiled smoother
    // dividers of a flat cell index (nc = n / 2, nq = n / 4, Ka the KL groups)
    FastDiv by_n, by_nc, by_nq, by_nn, by_ncnc, by_nnc, by_nnq, by_kan;
};

// Fill the dividers of level descriptor d (d.n set), on the host.
inline void set_divisors(LevelDesc& d, int Ka)
{
    const uint32_t n = static_cast<uint32_t>(d.n), nc = n / 2 > 0 ? n / 2 : 1, nq = n / 4 > 0 ? n / 4 : 1;
    d.by_n = FastDiv(n);
    d.by_nc = FastDiv(nc);
    d.by_nq = FastDiv(nq);
    d.by_nn = FastDiv(n * n);
    d.by_ncnc = FastDiv(nc * nc);
    d.by_nnc = FastDiv(n * nc);
    d.by_nnq = FastDiv(n * nq);
    d.by_kan = FastDiv(static_cast<uint32_t>(Ka > 0 ? Ka : 1) * n);
}

template <typename T>
struct Lv {
    int n;
    T* u;      // iterate (FMG solution on the current top level, correction below it)
    T* bc;     // right-hand side of the coarse correction equation
    T* kx;     // x faces: row i2, face f between cells f-1 and f, [i2*kx_pitch(n) + f]; f = 0, n hold 2k (boundary)
    T* ky;     // y faces: face g between rows g-1 and g, [g*n + i1]; g = 0, n hold 2k (boundary)
    T* idiag;  // 1 / (sum of the four face coefficients)
    T* k;      // coefficient exp(z) at the cell centres
    T* G;      // KL partial sums, Ka x n
    double* u64;  // mixed forms: FP64 solution
};

struct FmgArgs {
    const SampleDesc* samples;  // rank order: finest level descending
    int n_samples;
    const double* Y;  // normals, s per sample, indexed by canon
    const float* c32;  // mixed forms: sqrt(theta_m) y_m rounded to FP32, s per sample in rank order
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
    LevelDesc lv[MLQMC_MAX_LEVELS];
    ArrDesc chol;      // banded level-0 factor (FP64): entry q of sample i at base[q * stride + i] (elements)
    void* chol32;      // FP32 copy of the factor, same layout (mixed forms)
    double* F;         // F_t per rank, n_levels each
    double* usol;      // single-sample solutions (concatenated levels) or null
    int* queue;
    int* status;
    const int* active;  // per rank; null: all samples active
    double* norms;      // per rank residual norms
    int refine;         // solutions kept in u64 and corrected (mixed forms; converged FP64 form)
};

template <typename T>
__device__ __forceinline__ T* at(const ArrDesc& a, int i)
{
    return reinterpret_cast<T*>(a.base + static_cast<size_t>(i) * a.stride);
}

template <typename T>
__device__ __forceinline__ Lv<T> view(const FmgArgs& A, int t, int i)
{
    const LevelDesc& d = A.lv[t];
    Lv<T> L;
    L.n = d.n;
    L.u = at<T>(d.u, i);
    L.bc = at<T>(d.bc, i);
    L.kx = at<T>(d.kx, i);
    L.ky = at<T>(d.ky, i);
    L.idiag = at<T>(d.idiag, i);
    L.k = at<T>(d.k, i);
    L.G = at<T>(d.G, i);
    L.u64 = at<double>(d.u64, i);
    return L;
}

// A team of threads that works on one sample: a whole CTA or one warp.
struct BlockTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
    __device__ __forceinline__ bool first_warp() const { return threadIdx.x < 32; }
};

struct WarpTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool leader() const { return (threadIdx.x & 31) == 0; }
    __device__ __forceinline__ bool first_warp() const { return true; }
};

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

// Sum over the team, the same value in every thread, in a fixed order.
__device__ __forceinline__ double team_sum(const BlockTeam&, double v, double* red) { return block_sum(v, red); }

__device__ __forceinline__ double team_sum(const WarpTeam&, double v, double*)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 2^(j/64), j = 0..63, each rounded to the nearest double (table of exp64).
__device__ const double kExp2Tab[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0
};

// e^x in FP64 by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2),
// 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128 (ln2/64 split in two
// parts, the first with 32 significant bits, so that n ln2/64 subtracts
// exactly), e^x = 2^m 2^(j/64) e^r, e^r - 1 by its Taylor series to r^5
// (truncation below 4e-17 relative). Ten FP64 operations where the library
// exp takes about twice that on a part with GB300's FP64 rate. The lognormal
// fields keep |x| far below 700; beyond it the library exp answers.
static __device__ __noinline__ double exp_rare(double x) { return exp(x); }  // out of line: never if-converted

__device__ __forceinline__ double exp64(double x)
{
    if (!(fabs(x) < 700.0)) return exp_rare(x);
    constexpr double kMagic = 0x1.8p52;                  // 1.5 * 2^52: rounds to an integer in the low bits
    constexpr double kInvL = 0x1.71547652b82fep+6;       // 64 / ln2
    constexpr double kL1 = 0x1.62e42fee00000p-7;         // ln2/64, leading 32 bits
    constexpr double kL2 = 0x1.a39ef35793c76p-39;        // ln2/64 - kL1
    const double t = fma(x, kInvL, kMagic);
    const int n = __double2loint(t);
    const double kd = t - kMagic;
    double r = fma(-kd, kL1, x);
    r = fma(-kd, kL2, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    const double s = __ldg(&kExp2Tab[n & 63]);
    const double y = fma(s, q * r, s);
    return __longlong_as_double(__double_as_longlong(y) + (static_cast<long long>(n >> 6) << 52));
}

// 1/d for a positive normal d in FP64: the hardware's reciprocal estimate
// refined by two Newton-Raphson steps r <- r + r (1 - d r), each squaring the
// relative error, which ends within one ulp of the correctly rounded value
// in six FP64 operations (IEEE division takes about twelve).
__device__ __forceinline__ double rcp64(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// 1/sqrt(d) for a positive normal d in FP64: the hardware's estimate refined
// by two Newton-Raphson steps y <- y + (y/2)(1 - d y^2), each squaring the
// relative error, within about one ulp; eight FP64 operations in place of a
// square root and a division.
__device__ __forceinline__ double rsqrt64(double d)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double e = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    e = fma(-d * y, y, 1.0);
    return fma(0.5 * y, e, y);
}

__device__ __forceinline__ float expT(float x) { return expf(x); }
__device__ __forceinline__ double expT(double x) { return exp64(x); }

// Harmonic mean 2ab/(a+b) of two cell coefficients: FP32 with the hardware
// reciprocal (__fdividef, within 2 ulp; the coefficients are positive and
// far from the range where it flushes), FP64 through rcp64.
__device__ __forceinline__ float hmean(float a, float b) { return __fdividef(2.0f * a * b, a + b); }
__device__ __forceinline__ double hmean(double a, double b) { return 2.0 * a * b * rcp64(a + b); }
__device__ __forceinline__ float recip(float d) { return 1.0f / d; }
__device__ __forceinline__ double recip(double d) { return rcp64(d); }

// x face f of row i2 (f = 0..n) from the cell coefficients of that row.
template <typename T>
__device__ __forceinline__ T face_x(const T* k, int n, int i2, int f)
{
    const T* kr = k + i2 * n;
    if (f == 0) return T(2) * kr[0];
    if (f == n) return T(2) * kr[n - 1];
    return hmean(kr[f - 1], kr[f]);
}

// y face g of column i1 (g = 0..n).
template <typename T>
__device__ __forceinline__ T face_y(const T* k, int n, int g, int i1)
{
    if (g == 0) return T(2) * k[i1];
    if (g == n) return T(2) * k[(n - 1) * n + i1];
    return hmean(k[(g - 1) * n + i1], k[g * n + i1]);
}

template <typename T>
__device__ __forceinline__ T inv_diag(const T* kx, const T* ky, int n, int i1, int i2)
{
    const T* kr = kx + i2 * kx_pitch(n);
    return recip(kr[i1] + kr[i1 + 1] + ky[i2 * n + i1] + ky[(i2 + 1) * n + i1]);
}

// KL field on one level (eq. truncatedKL at the level's own cell centres):
// z(x1,x2) = sum_a psi_a(x1) G_a(x2), G_a(x2) = sum_{m: a_m = a} sqrt(theta_m) y_m psi_{b_m}(x2);
// then k = exp(z), harmonic-mean faces and the inverse diagonal.
template <typename T, typename TM>
__device__ void synth_level(const TM& tm, const FmgArgs& A, const Lv<T>& L, int t, const double* cy)
{
    const int n = L.n;
    const T* psi = static_cast<const T*>(A.psi) + A.psi_off[t];
    const int Ka = A.Ka;
    for (int idx = tm.rank(); idx < Ka * n; idx += tm.size()) {
        const int a = idx / n;
        const int i2 = idx - a * n;
        T acc = T(0);
        const int g1 = A.grp_start[a + 1];
        for (int g = A.grp_start[a]; g < g1; ++g) acc += static_cast<T>(cy[g]) * psi[A.grp_b[g] * n + i2];
        L.G[idx] = acc;
    }
    tm.sync();
    for (int p = tm.rank(); p < n * n; p += tm.size()) {
        const int i2 = p / n;
        const int i1 = p - i2 * n;
        T z = T(0);
        for (int a = 0; a < Ka; ++a) z += psi[a * n + i1] * L.G[a * n + i2];
        L.k[p] = expT(z);
    }
    tm.sync();
    for (int idx = tm.rank(); idx < n * (n + 1); idx += tm.size()) {
        const int i2 = idx / (n + 1);
        L.kx[i2 * kx_pitch(n) + idx - i2 * (n + 1)] = face_x(L.k, n, i2, idx - i2 * (n + 1));
        const int g = idx / n;
        L.ky[idx] = face_y(L.k, n, g, idx - g * n);
    }
    tm.sync();
    for (int p = tm.rank(); p < n * n; p += tm.size()) {
        const int i2 = p / n;
        L.idiag[p] = inv_diag(L.kx, L.ky, n, p - i2 * n, i2);
    }
    tm.sync();
}

// Gauss-Seidel update of one cell: u_P = (h^2 b_P + sum_Q k_PQ u_Q) / D_P.
template <typename T>
__device__ __forceinline__ void gs_cell(const Lv<T>& L, const T* b, T h2, int i1, int i2)
{
    const int n = L.n;
    const int p = i2 * n + i1;
    const T* kx = L.kx + i2 * kx_pitch(n);
    T acc = h2 * (b ? b[p] : T(1));
    if (i1 > 0) acc += kx[i1] * L.u[p - 1];
    if (i1 < n - 1) acc += kx[i1 + 1] * L.u[p + 1];
    if (i2 > 0) acc += L.ky[i2 * n + i1] * L.u[p - n];
    if (i2 < n - 1) acc += L.ky[(i2 + 1) * n + i1] * L.u[p + n];
    L.u[p] = acc * L.idiag[p];
}

// One red-black half sweep (colour 0: i1+i2 even). b == null: b = 1.
template <typename T, typename TM>
__device__ __forceinline__ void gs_colour(const TM& tm, const Lv<T>& L, const T* b, int colour)
{
    const int n = L.n;
    const int half = n >> 1;
    const T h2 = T(1) / (T(n) * T(n));
    for (int idx = tm.rank(); idx < n * half; idx += tm.size()) {
        const int i2 = idx / half;
        gs_cell(L, b, h2, 2 * (idx - i2 * half) + ((i2 + colour) & 1), i2);
    }
    tm.sync();
}

// (A u)_P scaled by h^2 in flux form: sum over faces k_f (u_P - u_Q), with
// u_Q = 0 across the boundary (where k_f holds 2 k_P). Differences of
// neighbouring values keep the FP64 residual floor near eps * |flux|.
template <typename T, typename U>
__device__ __forceinline__ U apply_h2(const T* kx, const T* ky, const U* u, int n, int i1, int i2)
{
    const int p = i2 * n + i1;
    const U up = u[p];
    U acc = U(kx[i2 * kx_pitch(n) + i1]) * (up - (i1 > 0 ? u[p - 1] : U(0)));
    acc += U(kx[i2 * kx_pitch(n) + i1 + 1]) * (up - (i1 < n - 1 ? u[p + 1] : U(0)));
    acc += U(ky[i2 * n + i1]) * (up - (i2 > 0 ? u[p - n] : U(0)));
    acc += U(ky[(i2 + 1) * n + i1]) * (up - (i2 < n - 1 ? u[p + n] : U(0)));
    return acc;
}

// Coarse value (I1, I2) of the restricted residual: mean over the 4 children of b - A u.
template <typename T>
__device__ __forceinline__ T resid_restrict_cell(const Lv<T>& F, const T* b, int I1, int I2)
{
    const int n = F.n;
    const T ih2 = T(n) * T(n);
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int i1 = 2 * I1 + (d & 1), i2 = 2 * I2 + (d >> 1);
        s += (b ? b[i2 * n + i1] : T(1)) - ih2 * apply_h2<T, T>(F.kx, F.ky, F.u, n, i1, i2);
    }
    return T(0.25) * s;
}

template <typename T, typename TM>
__device__ void resid_restrict(const TM& tm, const Lv<T>& F, const T* b, T* bc)
{
    const int nc = F.n >> 1;
    for (int idx = tm.rank(); idx < nc * nc; idx += tm.size()) {
        const int I2 = idx / nc;
        bc[idx] = resid_restrict_cell(F, b, idx - I2 * nc, I2);
    }
    tm.sync();
}

// Bilinear cell-centred prolongation (9,3,3,1)/16 of fine cell (i1, i2):
// 9/16 of the parent a, 3/16 of the coarse neighbours b (along x1) and c
// (along x2), 1/16 of the diagonal one d, with odd reflection across the
// Dirichlet boundary (a neighbour outside the grid is minus its mirror).
template <typename S, typename D>
__device__ __forceinline__ D prolong_cell(const S* e, int nc, int i1, int i2)
{
    const int I1 = i1 >> 1, I2 = i2 >> 1;
    const int J1 = (i1 & 1) ? I1 + 1 : I1 - 1;
    const int J2 = (i2 & 1) ? I2 + 1 : I2 - 1;
    const bool o1 = J1 < 0 || J1 >= nc, o2 = J2 < 0 || J2 >= nc;
    const int K1 = o1 ? I1 : J1, K2 = o2 ? I2 : J2;
    const D a = D(e[I2 * nc + I1]);
    const D b0 = D(e[I2 * nc + K1]);
    const D c0 = D(e[K2 * nc + I1]);
    const D d0 = D(e[K2 * nc + K1]);
    const D b = o1 ? -b0 : b0;
    const D c = o2 ? -c0 : c0;
    const D d = (o1 != o2) ? -d0 : d0;
    return fma(D(0.5625), a, fma(D(0.1875), b + c, D(0.0625) * d));
}

template <typename S, typename D, bool ADD, typename TM>
__device__ void prolong(const TM& tm, const S* e, int nc, D* fine)
{
    const int nf = 2 * nc;
    for (int p = tm.rank(); p < nf * nf; p += tm.size()) {
        const int i2 = p / nf;
        const D v = prolong_cell<S, D>(e, nc, p - i2 * nf, i2);
        if (ADD) fine[p] += v;
        else fine[p] = v;
    }
    tm.sync();
}

// Banded Cholesky of h0^2 A_0 (bandwidth n0) by the team's first warp:
// Lb[i*(n0+1) + d] = L(i, i-d).
template <typename F, typename TM>
__device__ void chol_factor(const TM& tm, double* Lb, int n0, const F* kx, const F* ky)
{
    if (tm.first_warp()) {
        const int N = n0 * n0, W = n0 + 1, lane = threadIdx.x & 31;
        for (int j = 0; j < N; ++j) {
            const int j1 = j % n0, j2 = j / n0;
            double d = static_cast<double>(kx[j2 * kx_pitch(n0) + j1]) + static_cast<double>(kx[j2 * kx_pitch(n0) + j1 + 1]) +
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
                if (lane == 1 && i1 > 0) a = -static_cast<double>(kx[i2 * kx_pitch(n0) + i1]);
                if (lane == n0) a = -static_cast<double>(ky[i2 * n0 + i1]);
                for (int tt = (i - n0 > 0 ? i - n0 : 0); tt < j; ++tt) a -= Lb[i * W + (i - tt)] * Lb[j * W + (j - tt)];
                Lb[i * W + lane] = a / Ljj;
            }
            __syncwarp();
        }
    }
    tm.sync();
}

// Solve (h0^2 A_0) x = h0^2 b with the band factor, in the factor's precision
// F; b == null: b = 1. Team leader.
template <typename B, typename X, typename F, typename TM>
__device__ void chol_solve(const TM& tm, const F* Lb, int n0, const B* b, X* x, F* tmp)
{
    if (tm.leader()) {
        const int N = n0 * n0, W = n0 + 1;
        const F h2 = F(1) / (F(n0) * F(n0));
        for (int i = 0; i < N; ++i) {
            F v = h2 * (b ? static_cast<F>(b[i]) : F(1));
            for (int q = 1; q <= n0 && q <= i; ++q) v -= Lb[i * W + q] * tmp[i - q];
            tmp[i] = v / Lb[i * W];
        }
        for (int i = N - 1; i >= 0; --i) {
            F v = tmp[i];
            for (int q = 1; q <= n0 && i + q < N; ++q) v -= Lb[(i + q) * W + q] * tmp[i + q];
            tmp[i] = v / Lb[i * W];
        }
        for (int i = 0; i < N; ++i) x[i] = static_cast<X>(tmp[i]);
    }
    tm.sync();
}

template <typename T, typename TM>
__device__ void zero(const TM& tm, T* a, int cnt)
{
    for (int p = tm.rank(); p < cnt; p += tm.size()) a[p] = T(0);
    tm.sync();
}

// V-cycle (Sec. 4 correction scheme, recursively) of sample i on levels
// t_top..0. top_b == null: right-hand side 1 on the top level; the top
// iterate is used as given, lower levels start from zero. The exact level-0
// solve uses the band factor Lb in the working precision T.
template <typename T, typename TM>
__device__ void vcycle(const TM& tm, const FmgArgs& A, int i, int t_top, const T* top_b, const T* Lb, T* tmp)
{
    for (int t = t_top; t >= 1; --t) {
        const Lv<T> F = view<T>(A, t, i);
        const T* b = (t == t_top) ? top_b : F.bc;
        if (t < t_top) zero(tm, F.u, F.n * F.n);
        for (int s = 0; s < A.nu1; ++s) {
            gs_colour(tm, F, b, 0);
            gs_colour(tm, F, b, 1);
        }
        resid_restrict(tm, F, b, view<T>(A, t - 1, i).bc);
    }
    {
        const Lv<T> C0 = view<T>(A, 0, i);
        chol_solve(tm, Lb, A.n0, t_top == 0 ? top_b : C0.bc, C0.u, tmp);
    }
    for (int t = 1; t <= t_top; ++t) {
        const Lv<T> F = view<T>(A, t, i);
        const Lv<T> Cl = view<T>(A, t - 1, i);
        prolong<T, T, true>(tm, Cl.u, Cl.n, F.u);
        const T* b = (t == t_top) ? top_b : F.bc;
        for (int s = 0; s < A.nu2; ++s) {
            gs_colour(tm, F, b, 1);
            gs_colour(tm, F, b, 0);
        }
    }
}

// Exact widening of a positive normal float (a face coefficient) to double by
// re-biasing its exponent on the integer pipe: the 8-bit exponent e becomes
// e - 127 + 1023 and the 23-bit mantissa moves to the top of the 52-bit one.
__device__ __forceinline__ double widen_pos(float f)
{
    const unsigned long long b = static_cast<unsigned long long>(__float_as_uint(f) & 0x7FFFFFFFu);
    return __longlong_as_double(static_cast<long long>((b << 29) + (896ull << 52)));
}
__device__ __forceinline__ double widen_pos(double f) { return f; }

// The conversion instructions, kept out of line: when the compiler turns a
// short two-way branch into a select it issues both sides, and these belong
// to the FP64 pipe on GB300; a call runs only for the lanes that take it.
static __device__ __noinline__ double widen_rare(float f) { return static_cast<double>(f); }
static __device__ __noinline__ float narrow_rare(double x) { return __double2float_rn(x); }

// float -> double (exact) by moving the bits: sign, exponent rebiased by
// 1023 - 127, mantissa shifted up by 29; zero by a select. Subnormal,
// infinite and NaN inputs take the conversion instruction (out of line).
__device__ __forceinline__ double widen(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t mag = b & 0x7FFFFFFFu;
    const unsigned long long sgn = static_cast<unsigned long long>(b & 0x80000000u) << 32;
    if (mag == 0u) return __longlong_as_double(static_cast<long long>(sgn));
    if (mag - 0x00800000u >= 0x7F000000u) return widen_rare(f);
    return __longlong_as_double(static_cast<long long>(sgn | ((static_cast<unsigned long long>(mag) << 29) + (896ull << 52))));
}
__device__ __forceinline__ double widen(double f) { return f; }

// double -> float rounded to nearest even, in integer arithmetic on the bits
// when the result is a normal float or overflows (biased exponent of |x| in
// 897..1150): add 2^28 - 1 plus the lowest kept bit, drop 29 mantissa bits,
// rebias the exponent (a carry out of the mantissa moves into the exponent,
// up to infinity); zero by a select. Smaller magnitudes, infinities and NaN
// take the conversion instruction (out of line).
__device__ __forceinline__ float narrow(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t sgn = static_cast<uint32_t>(b >> 32) & 0x80000000u;
    if (a == 0ull) return __uint_as_float(sgn);
    const unsigned e = static_cast<unsigned>(a >> 52);
    if (e < 897u || e > 1150u) return narrow_rare(x);
    const unsigned long long r = a + 0x0FFFFFFFull + ((a >> 29) & 1ull);
    const uint32_t mag = static_cast<uint32_t>((r >> 29) - (896ull << 23));
    return __uint_as_float(mag | sgn);
}

static __device__ __noinline__ float narrow_rest_rare(double x, float hi)
{
    return __double2float_rn(x - static_cast<double>(hi));
}

// x - narrow(x) rounded to FP32, from the bits of x: the 29 significand bits
// that narrow() drops, less 2^29 when it rounded up, times 2^(e - 1075) (e the
// biased exponent of x); exact before that last rounding, which errs by at
// most 2^-48 |x|. Exponents below 949 (|x| < 2^-74) or outside narrow()'s
// integer path take an FP64 subtraction (out of line).
__device__ __forceinline__ float narrow_rest(double x, float hi)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned e = static_cast<unsigned>(a >> 52);
    if (e < 949u || e > 1150u) return narrow_rest_rare(x, hi);
    const uint32_t low = static_cast<uint32_t>(a & 0x1FFFFFFFull);
    const uint32_t up = (low + 0x0FFFFFFFu + (static_cast<uint32_t>(a >> 29) & 1u)) >> 29;
    const int d = static_cast<int>(low) - static_cast<int>(up << 29);
    const float mag = static_cast<float>(d) * __uint_as_float((e - 948u) << 23);
    return (b >> 63) ? -mag : mag;
}

// Running sum of FP64 values given as FP32 pairs (hi, lo), x = hi + lo: hi
// added by TwoSum (the rounding error kept), the errors and the lo parts
// added in FP32. For k values the error is within about k 2^-48 of their
// magnitudes' sum, without the FP64 pipe.
struct PairSum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float h, float l)
    {
        const float s = hi + h;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (h - bb)) + l;
        hi = s;
    }
    __device__ __forceinline__ double value() const { return widen(hi) + widen(lo); }
};

// Error-free transformations in FP32: Knuth's TwoSum (a + b = s + e exactly)
// and the product error by one FMA (a b = p + e exactly), the building blocks
// of compensated sums and dot products (Ogita, Rump and Oishi, SIAM J. Sci.
// Comput. 26, 2005). The round-to-nearest intrinsics keep the compiler from
// contracting or reassociating them.
__device__ __forceinline__ void two_sum32(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// r = 1 - c sum_j k_j (u_P - u_j) for FP32 inputs, c = n^2 (exact in FP32),
// rounded once to FP32: each difference exactly as a pair (TwoSum), each
// product as a pair (FMA error), the four pairs summed with TwoSum on the
// leading parts and the trailing parts accumulated (the cascaded summation
// Sum2 of Ogita, Rump and Oishi), the scaling by c as a pair. Before the
// final rounding the error is a few units of 2^-48 of c sum_j |k_j (u_P - u_j)|,
// below the FP32 rounding of r unless the terms cancel by more than 2^20.
// All on the FP32 pipe (about 70 operations in place of 9 FP64 ones).
__device__ __forceinline__ float resid_f32x2(const float (&k)[4], float up, const float (&u)[4], float c)
{
    float ph[4], pl[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float dh, dl;
        two_sum32(up, -u[j], dh, dl);
        ph[j] = __fmul_rn(k[j], dh);
        pl[j] = __fmaf_rn(k[j], dl, __fmaf_rn(k[j], dh, -ph[j]));
    }
    float sh = ph[0], sl = pl[0];
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        float e;
        two_sum32(sh, ph[j], sh, e);
        sl = __fadd_rn(sl, __fadd_rn(e, pl[j]));
    }
    const float ah = __fmul_rn(c, sh);
    const float al = __fmaf_rn(c, sl, __fmaf_rn(c, sh, -ah));
    float rh, re;
    two_sum32(1.0f, -ah, rh, re);
    return __fadd_rn(rh, __fsub_rn(re, al));
}

// The mixed forms' one refinement update of a cell, u64 + e: in the fixed-
// cycle forms u64 still holds the widened FP32 interpolant U, so U + e is a
// sum of two floats that TwoSum gives exactly as the pair (h, lo): h =
// fl32(U + e) is the FP32 copy and (h, lo) goes into a PairSum; the FP64
// value h + lo (the correctly rounded U + e, as the FP64 add gives it) is
// formed only when it is stored (keep). A u64 that is not a widened float
// takes the FP64 add.
__device__ __forceinline__ void update_pair(double w, float e, bool keep, float& h, float& lo, double& r)
{
    const float U = narrow(w);
    if (__double_as_longlong(widen(U)) == __double_as_longlong(w)) {
        two_sum32(U, e, h, lo);
        if (keep) r = widen(h) + widen(lo);
    } else {
        r = w + widen(e);
        h = narrow(r);
        lo = narrow_rest(r, h);
    }
}

// A double result stored in working precision T.
template <typename T>
__device__ __forceinline__ T to_work(double x)
{
    if constexpr (sizeof(T) == 4) return narrow(x);
    else return x;
}

// (A u)_P h^2 in flux form, FP64, from working-precision faces.
template <typename T>
__device__ __forceinline__ double apply_h2_64(const T* kx, const T* ky, const double* u, int n, int i1, int i2)
{
    const int p = i2 * n + i1;
    const double up = u[p];
    double acc = widen_pos(kx[i2 * kx_pitch(n) + i1]) * (up - (i1 > 0 ? u[p - 1] : 0.0));
    acc = fma(widen_pos(kx[i2 * kx_pitch(n) + i1 + 1]), up - (i1 < n - 1 ? u[p + 1] : 0.0), acc);
    acc = fma(widen_pos(ky[i2 * n + i1]), up - (i2 > 0 ? u[p - n] : 0.0), acc);
    acc = fma(widen_pos(ky[(i2 + 1) * n + i1]), up - (i2 < n - 1 ? u[p + n] : 0.0), acc);
    return acc;
}

// Refinement path (mixed forms, and the converged FP64 form): r = 1 - A u64 of
// one cell in FP64 with the working-precision faces widened; ih2 = n^2,
// hoisted by the caller.
template <typename T>
__device__ __forceinline__ double resid64_cell(const Lv<T>& L, double ih2, int i1, int i2)
{
    return fma(-ih2, apply_h2_64<T>(L.kx, L.ky, L.u64, L.n, i1, i2), 1.0);
}

template <typename T, typename TM>
__device__ double qoi(const TM& tm, const T* u, int n, int kind, double* red)
{
    if (kind == MLQMC_QOI_MEAN) {
        double acc = 0.0;
        for (int p = tm.rank(); p < n * n; p += tm.size()) acc += static_cast<double>(u[p]);
        return team_sum(tm, acc, red) / (static_cast<double>(n) * n);
    }
    const int m = n / 2;
    const double v = 0.25 * (static_cast<double>(u[(m - 1) * n + (m - 1)]) + static_cast<double>(u[(m - 1) * n + m]) +
                             static_cast<double>(u[m * n + (m - 1)]) + static_cast<double>(u[m * n + m]));
    tm.sync();
    return v;
}

template <typename T, typename TM>
__device__ void copy_out(const TM& tm, const T* src, double* dst, int cnt)
{
    for (int p = tm.rank(); p < cnt; p += tm.size()) dst[p] = static_cast<double>(src[p]);
    tm.sync();
}

}  // namespace mlqmc_dev
