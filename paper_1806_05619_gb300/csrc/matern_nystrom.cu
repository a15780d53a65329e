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

// Matern covariance at distance r (eq. matern) for nu = 1/2, 3/2, 5/2, where
// 2^(1-nu)/Gamma(nu) z^nu K_nu(z) reduces to exp(-z) times 1, (1 + z) and
// (1 + z + z^2/3) with z = sqrt(2 nu) r / corr_len.
__host__ __device__ inline double matern_cov(double r, int code, double lam, double sig2)
{
    if (code == 0) {
        const double z = r / lam;
        return sig2 * exp(-z);
    }
    if (code == 1) {
        const double z = 1.7320508075688772 * r / lam;  // sqrt(3)
        return sig2 * (1.0 + z) * exp(-z);
    }
    const double z = 2.23606797749979 * r / lam;  // sqrt(5)
    return sig2 * (1.0 + z + z * z / 3.0) * exp(-z);
}

int nu_code(double nu)
{
    return nu == 0.5 ? 0 : (nu == 1.5 ? 1 : 2);
}

// B[k][q] = w C(|x_k - x_q|), node q = (q % m, q / m), x = ((i + 1/2)/m).
__global__ void kb_nystrom_matrix(int m, int code, double lam, double sig2, double* B)
{
    const int64_t M = static_cast<int64_t>(m) * m;
    const double w = 1.0 / (static_cast<double>(m) * m);
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < M * M;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(e / M), q = static_cast<int>(e - static_cast<int64_t>(k) * M);
        const double dx = static_cast<double>(k % m - q % m) / m, dy = static_cast<double>(k / m - q / m) / m;
        B[e] = w * matern_cov(sqrt(dx * dx + dy * dy), code, lam, sig2);
    }
}

constexpr int kCells = 64;   // cells per CTA
constexpr int kModes = 64;   // modes per CTA
constexpr int kNodes = 32;   // nodes per shared-memory chunk
constexpr int kThreads = 256;

// out[p][j] = sum_q C(|x_p - x_q|) wpsi[q][j] for the CTA's 64 cells x 64
// modes: covariance tile (64 cells x 32 nodes) and weight tile (32 nodes x 64
// modes) in shared memory; thread (c, g) accumulates cell c, modes 16g..16g+15.
__global__ void __launch_bounds__(kThreads) kb_nystrom_interp(int n, int m, int code, double lam, double sig2, int s,
                                                              const double* __restrict__ wpsi, double* __restrict__ out)
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
                v = matern_cov(sqrt(dx * dx + dy * dy), code, lam, sig2);
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
    return nu == 0.5 || nu == 1.5 || nu == 2.5;
}

mlqmc_status nodal_modes(double nu, double corr_len, double sigma, int m, int s, double* theta, double* psi)
{
    if (!supported_nu(nu) || !(corr_len > 0.0) || !(sigma > 0.0) || m < 2 || m > 128 || s < 1 || s > m * m ||
        !theta || !psi)
        return MLQMC_ERR_INVALID_ARG;
    const int M = m * m;
    double *dB = nullptr, *dW = nullptr, *dwork = nullptr;
    int* dinfo = nullptr;
    cusolverDnHandle_t h = nullptr;
    mlqmc_status st = MLQMC_OK;
    int lwork = 0, info = 0;
    std::vector<double> evals(M), vecs;
    if (cudaMalloc(&dB, sizeof(double) * M * M) != cudaSuccess || cudaMalloc(&dW, sizeof(double) * M) != cudaSuccess ||
        cudaMalloc(&dinfo, sizeof(int)) != cudaSuccess) {
        st = MLQMC_ERR_OOM;
        goto done;
    }
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) {
        st = MLQMC_ERR_CUDA;
        goto done;
    }
    {
        const int64_t tot = static_cast<int64_t>(M) * M;
        const int grid = static_cast<int>(std::min<int64_t>((tot + 255) / 256, 152 * 64));
        kb_nystrom_matrix<<<grid, 256>>>(m, nu_code(nu), corr_len, sigma * sigma, dB);
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
    return st;
}

bool interpolate(double nu, double corr_len, double sigma, int m, int s, const double* d_wpsi, int n, double* d_out,
                 cudaStream_t st)
{
    const int64_t ncell = static_cast<int64_t>(n) * n;
    dim3 grid(static_cast<unsigned>((ncell + kCells - 1) / kCells), static_cast<unsigned>((s + kModes - 1) / kModes));
    kb_nystrom_interp<<<grid, kThreads, 0, st>>>(n, m, nu_code(nu), corr_len, sigma * sigma, s, d_wpsi, d_out);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mlqmc_matern

extern "C" mlqmc_status mlqmc_nystrom_modes(double nu, double corr_len, double sigma, int32_t m, int32_t s,
                                            double* theta_out, double* psi_out)
{
    return mlqmc_matern::nodal_modes(nu, corr_len, sigma, m, s, theta_out, psi_out);
}
