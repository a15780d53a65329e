// Matern covariance (eq. matern) and its Nystrom eigenpairs (Sec. 5).
#pragma once

#include <cuda_runtime.h>

#include "mlqmc.h"

namespace mlqmc_matern {

// nu in {0.5, 1, 1.5, 2, 2.5}: half-integer orders in closed form, 1 and 2 by quadrature.
bool supported_nu(double nu);

// The s largest Nystrom eigenpairs on the m x m midpoint nodes (see
// mlqmc_nystrom_modes): theta (s, descending), psi (m*m x s, node-major,
// sum_q w_q psi_j(x_q)^2 = 1). Host outputs; blocking.
mlqmc_status nodal_modes(double nu, double corr_len, double sigma, int m, int s, double* theta, double* psi);

// Psi_t(x_p, j) = 1/theta_j sum_q w_q C(x_p, x_q) psi_j(x_q) at the n x n cell
// centres (Nystrom interpolation formula, Sec. 5), FP64, cell-major
// (d_out[p * s + j]). d_wpsi: device, m*m x s, w_q psi_j(x_q) / theta_j.
bool interpolate(double nu, double corr_len, double sigma, int m, int s, const double* d_wpsi, int n,
                 double* d_out, cudaStream_t st);

}  // namespace mlqmc_matern
