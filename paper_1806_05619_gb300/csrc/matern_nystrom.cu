// Matern covariance (eq. matern) and its Nystrom eigenpairs (Sec. 5: the
// integral eigenproblem eq. inteq collocated at quadrature nodes, eqs.
// discrinteq and matrixequation, and the Nystrom interpolation formula).
//
// Nodes: the cell centres of an m x m grid on the unit square, midpoint
// weights w = 1/m^2. The symmetric form B = sqrt(W) Sigma sqrt(W) = w Sigma
// is built on the device and handed to cuSOLVER's dense symmetric
// eigensolver (a set-up step, run once per problem, not per sample). The
// interpolation to a level's cell centres is a dense contraction over the
// nodes with the covariance generated on the fly, tiled through shared
// memory; it runs once per level at context creation.
#include "matern_nystrom.h"

#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// Covariance of one problem: code 0, 1, 2 for nu = 1/2, 3/2, 5/2 (closed
// forms); 3, 4 for nu = 1, 2 (a table of C and dC/dr at r_k = k h with cubic
// Hermite interpolation, and direct evaluation for z below kZDirect).
struct Cov {
    int code;
    double lam, sig2;
    const double* tab;  // integer nu: (C, dC/dr) pairs, ntab of them
    double h;
    int ntab;
};

constexpr int kTab = (1 << 18) + 1;
constexpr double kZDirect = 0.01;

// z^nu K_nu(z), integer nu >= 0, z > 0: the trapezoidal rule with step 1/4 on
// K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt. The integrand is analytic
// in the strip |Im t| < pi/2, so the rule's error falls like exp(-pi^2 / step)
// (below 1e-17 here; Trefethen and Weideman, SIAM Review 56, 2014); terms are
// added until they are below 1e-18 of the sum past the integrand's peak.
__device__ double zk_trap(int nu, double z)
{
    constexpr double tau = 0.25;
    double sum = 0.5 * exp(-z);
    for (int k = 1; k < 600; ++k) {
        const double t = k * tau;
        const double et = exp(t);
        const double ch = 0.5 * (et + 1.0 / et);
        const double cn = nu == 0 ? 1.0 : 0.5 * (exp(nu * t) + exp(-nu * t));
        const double term = exp(-z * ch) * cn;
        sum += term;
        if (term < 1e-18 * sum && z * ch > nu * t + 40.0) break;
    }
    double zn = 1.0;
    for (int q = 0; q < nu; ++q) zn *= z;
    return zn * tau * sum;
}

// Matern covariance at distance r (eq. matern). nu = 1/2, 3/2, 5/2:
// 2^(1-nu)/Gamma(nu) z^nu K_nu(z) reduces to exp(-z) times 1, (1 + z) and
// (1 + z + z^2/3), z = sqrt(2 nu) r / corr_len. nu = 1, 2: 2^(1-nu) z^nu K_nu(z)
// (Gamma(1) = Gamma(2) = 1) from the table, or directly for small z.
__device__ double matern_cov(double r, const Cov& cv)
{
    if (cv.code == 0) {
        const double z = r / cv.lam;
        return cv.sig2 * exp(-z);
    }
    if (cv.code == 1) {
        const double z = 1.7320508075688772 * r / cv.lam;  // sqrt(3)
        return cv.sig2 * (1.0 + z) * exp(-z);
    }
    if (cv.code == 2) {
        const double z = 2.23606797749979 * r / cv.lam;  // sqrt(5)
        return cv.sig2 * (1.0 + z + z * z / 3.0) * exp(-z);
    }
    const int nu = cv.code - 2;
    const double z = sqrt(2.0 * nu) * r / cv.lam;
    if (z < kZDirect) {
        if (z == 0.0) return cv.sig2;
        return cv.sig2 * (nu == 1 ? 1.0 : 0.5) * zk_trap(nu, z);
    }
    const double sr = r / cv.h;
    int k = static_cast<int>(sr);
    if (k > cv.ntab - 2) k = cv.ntab - 2;
    const double t = sr - k, t2 = t * t, t3 = t2 * t;
    const double* a = cv.tab + 2 * k;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * a[0] + (t3 - 2.0 * t2 + t) * cv.h * a[1] + (-2.0 * t3 + 3.0 * t2) * a[2] +
           (t3 - t2) * cv.h * a[3];
}

// Table for integer nu: C(r_k) and dC/dr(r_k), r_k = k h, from
// d/dz [z^nu K_nu(z)] = -z^nu K_(nu-1)(z) = -z (z^(nu-1) K_(nu-1)(z)).
__global__ void kb_matern_table(int nu, double lam, double sig2, double h, int ntab, double* tab)
{
    const double c = nu == 1 ? 1.0 : 0.5, dz = sqrt(2.0 * nu) / lam;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ntab; k += gridDim.x * blockDim.x) {
        const double z = dz * k * h;
        if (k == 0) {
            tab[0] = sig2;
            tab[1] = 0.0;
            continue;
        }
        tab[2 * k] = sig2 * c * zk_trap(nu, z);
        tab[2 * k + 1] = -sig2 * c * z * zk_trap(nu - 1, z) * dz;
    }
}

int nu_code(double nu)
{
    return nu == 0.5 ? 0 : nu == 1.5 ? 1 : nu == 2.5 ? 2 : nu == 1.0 ? 3 : 4;
}

// Device covariance of (nu, corr_len, sigma); integer nu builds its table in *d_tab (caller frees).
bool make_cov(double nu, double lam, double sigma, Cov* cv, double** d_tab, cudaStream_t st)
{
    cv->code = nu_code(nu);
    cv->lam = lam;
    cv->sig2 = sigma * sigma;
    cv->tab = nullptr;
    cv->ntab = kTab;
    cv->h = 1.4143 / (kTab - 1);  // r up to the unit square's diagonal
    *d_tab = nullptr;
    if (cv->code < 3) return true;
    if (cudaMalloc(d_tab, sizeof(double) * 2 * kTab) != cudaSuccess) return false;
    kb_matern_table<<<(kTab + 255) / 256, 256, 0, st>>>(cv->code - 2, lam, cv->sig2, cv->h, kTab, *d_tab);
    cv->tab = *d_tab;
    return cudaGetLastError() == cudaSuccess;
}

// B[k][q] = w C(|x_k - x_q|), node q = (q % m, q / m), x = ((i + 1/2)/m).
__global__ void kb_nystrom_matrix(int m, Cov cv, double* B)
{
    const int64_t M = static_cast<int64_t>(m) * m;
    const double w = 1.0 / (static_cast<double>(m) * m);
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < M * M;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(e / M), q = static_cast<int>(e - static_cast<int64_t>(k) * M);
        const double dx = static_cast<double>(k % m - q % m) / m, dy = static_cast<double>(k / m - q / m) / m;
        B[e] = w * matern_cov(sqrt(dx * dx + dy * dy), cv);
    }
}

constexpr int kCells = 64;   // cells per CTA
constexpr int kModes = 64;   // modes per CTA
constexpr int kNodes = 32;   // nodes per shared-memory chunk
constexpr int kThreads = 256;

// out[p][j] = sum_q C(|x_p - x_q|) wpsi[q][j] for the CTA's 64 cells x 64
// modes: covariance tile (64 cells x 32 nodes) and weight tile (32 nodes x 64
// modes) in shared memory; thread (c, g) accumulates cell c, modes 16g..16g+15.
__global__ void __launch_bounds__(kThreads) kb_nystrom_interp(int n, int m, Cov cv, int s, const double* __restrict__ wpsi,
                                                              double* __restrict__ out)
{
    __shared__ double Ct[kCells][kNodes + 1];
    __shared__ double Wt[kNodes][kModes];
    const int64_t ncell = static_cast<int64_t>(n) * n;
    const int M = m * m;
    const int c = threadIdx.x % kCells, g = threadIdx.x / kCells;
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kCells;
    const int j0 = blockIdx.y * kModes;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int q0 = 0; q0 < M; q0 += kNodes) {
        for (int e = threadIdx.x; e < kCells * kNodes; e += kThreads) {
            const int cc = e / kNodes, qq = e % kNodes;
            const int64_t p = p0 + cc;
            const int q = q0 + qq;
            double v = 0.0;
            if (p < ncell && q < M) {
                const int i2 = static_cast<int>(p / n), i1 = static_cast<int>(p - static_cast<int64_t>(i2) * n);
                const double dx = (i1 + 0.5) / n - (q % m + 0.5) / m, dy = (i2 + 0.5) / n - (q / m + 0.5) / m;
                v = matern_cov(sqrt(dx * dx + dy * dy), cv);
            }
            Ct[cc][qq] = v;
        }
        for (int e = threadIdx.x; e < kNodes * kModes; e += kThreads) {
            const int qq = e / kModes, jj = e % kModes;
            const int q = q0 + qq, j = j0 + jj;
            Wt[qq][jj] = (q < M && j < s) ? wpsi[static_cast<size_t>(q) * s + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int qq = 0; qq < kNodes; ++qq) {
            const double cq = Ct[c][qq];
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = fma(cq, Wt[qq][g * 16 + k], acc[k]);
        }
        __syncthreads();
    }
    const int64_t p = p0 + c;
    if (p < ncell) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int j = j0 + g * 16 + k;
            if (j < s) out[p * s + j] = acc[k];
        }
    }
}

}  // namespace

namespace mlqmc_matern {

bool supported_nu(double nu)
{
    return nu == 0.5 || nu == 1.5 || nu == 2.5 || nu == 1.0 || nu == 2.0;
}

mlqmc_status nodal_modes(double nu, double corr_len, double sigma, int m, int s, double* theta, double* psi)
{
    if (!supported_nu(nu) || !(corr_len > 0.0) || !(sigma > 0.0) || m < 2 || m > 128 || s < 1 || s > m * m ||
        !theta || !psi)
        return MLQMC_ERR_INVALID_ARG;
    const int M = m * m;
    double *dB = nullptr, *dW = nullptr, *dwork = nullptr, *dtab = nullptr;
    int* dinfo = nullptr;
    Cov cv{};
    cusolverDnHandle_t h = nullptr;
    mlqmc_status st = MLQMC_OK;
    int lwork = 0, info = 0;
    std::vector<double> evals(M), vecs;
    if (cudaMalloc(&dB, sizeof(double) * M * M) != cudaSuccess || cudaMalloc(&dW, sizeof(double) * M) != cudaSuccess ||
        cudaMalloc(&dinfo, sizeof(int)) != cudaSuccess) {
        st = MLQMC_ERR_OOM;
        goto done;
    }
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS || !make_cov(nu, corr_len, sigma, &cv, &dtab, 0)) {
        st = MLQMC_ERR_CUDA;
        goto done;
    }
    {
        const int64_t tot = static_cast<int64_t>(M) * M;
        const int grid = static_cast<int>(std::min<int64_t>((tot + 255) / 256, 152 * 64));
        kb_nystrom_matrix<<<grid, 256>>>(m, cv, dB);
        if (cudaGetLastError() != cudaSuccess) {
            st = MLQMC_ERR_CUDA;
            goto done;
        }
    }
    if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, dB, M, dW, &lwork) !=
        CUSOLVER_STATUS_SUCCESS) {
        st = MLQMC_ERR_CUDA;
        goto done;
    }
    if (cudaMalloc(&dwork, sizeof(double) * std::max(1, lwork)) != cudaSuccess) {
        st = MLQMC_ERR_OOM;
        goto done;
    }
    if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, dB, M, dW, dwork, lwork, dinfo) !=
            CUSOLVER_STATUS_SUCCESS ||
        cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || info != 0) {
        st = MLQMC_ERR_CUDA;
        goto done;
    }
    vecs.resize(static_cast<size_t>(M) * M);
    if (cudaMemcpy(evals.data(), dW, sizeof(double) * M, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(vecs.data(), dB, sizeof(double) * M * M, cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = MLQMC_ERR_CUDA;
        goto done;
    }
    // ascending from the solver; column i of the column-major result is eigenvector i
    for (int j = 0; j < s; ++j) {
        const int i = M - 1 - j;
        theta[j] = evals[i];
        for (int q = 0; q < M; ++q) psi[static_cast<size_t>(q) * s + j] = vecs[static_cast<size_t>(i) * M + q] * m;
    }
done:
    if (h) cusolverDnDestroy(h);
    cudaFree(dB);
    cudaFree(dW);
    cudaFree(dwork);
    cudaFree(dinfo);
    cudaFree(dtab);
    return st;
}

bool interpolate(double nu, double corr_len, double sigma, int m, int s, const double* d_wpsi, int n, double* d_out,
                 cudaStream_t st)
{
    const int64_t ncell = static_cast<int64_t>(n) * n;
    Cov cv{};
    double* dtab = nullptr;
    bool good = make_cov(nu, corr_len, sigma, &cv, &dtab, st);
    if (good) {
        dim3 grid(static_cast<unsigned>((ncell + kCells - 1) / kCells),
                  static_cast<unsigned>((s + kModes - 1) / kModes));
        kb_nystrom_interp<<<grid, kThreads, 0, st>>>(n, m, cv, s, d_wpsi, d_out);
        good = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    }
    cudaFree(dtab);
    return good;
}

}  // namespace mlqmc_matern

extern "C" mlqmc_status mlqmc_nystrom_modes(double nu, double corr_len, double sigma, int32_t m, int32_t s,
                                            double* theta_out, double* psi_out)
{
    return mlqmc_matern::nodal_modes(nu, corr_len, sigma, m, s, theta_out, psi_out);
}
