"""Oracle for the Matern covariance and its Nystrom eigenpairs (Sec. 5: eq.
inteq collocated at quadrature nodes, eqs. discrinteq and matrixequation, the
Nystrom interpolation formula; eq. matern). Plain numpy/scipy in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only ``tests/`` may
import it. Library routines serve as steps: ``numpy.linalg.eigh`` for the
symmetric eigenproblem and ``scipy.special.kv``/``gamma`` for the Bessel form
of eq. matern. Nodes: the cell centres of an m x m grid (q = k2*m + k1) with
midpoint weights 1/m^2 (reading A29).
"""
from __future__ import annotations

import numpy as np


def matern_bessel(r, nu, corr_len, sigma=1.0):
    """eq. matern as printed: 2^(1-nu)/Gamma(nu) (sqrt(2 nu) rho)^nu K_nu(sqrt(2 nu) rho),
    rho = r / corr_len, times sigma^2; 1 at r = 0."""
    from scipy.special import gamma, kv

    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r / corr_len
    with np.errstate(invalid="ignore", divide="ignore"):
        v = 2.0 ** (1.0 - nu) / gamma(nu) * z ** nu * kv(nu, z)
    return sigma ** 2 * np.where(z == 0.0, 1.0, v)


def matern(r, nu, corr_len, sigma=1.0):
    """eq. matern: for nu = 1/2, 3/2, 5/2 in closed form (K_nu of half-integer
    order): exp(-z) times 1, 1 + z, 1 + z + z^2/3, z = sqrt(2 nu) r / corr_len;
    for nu = 1, 2 the Bessel form."""
    if nu in (1.0, 2.0):
        return matern_bessel(r, nu, corr_len, sigma)
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r / corr_len
    if nu == 0.5:
        p = 1.0
    elif nu == 1.5:
        p = 1.0 + z
    elif nu == 2.5:
        p = 1.0 + z + z * z / 3.0
    else:
        raise ValueError("closed forms for nu in {0.5, 1.5, 2.5}")
    return sigma ** 2 * p * np.exp(-z)


def nodes(m):
    """Midpoint nodes of the unit square, q = k2*m + k1: (x1, x2) arrays, weight 1/m^2."""
    k = (np.arange(m) + 0.5) / m
    x1 = np.tile(k, m)
    x2 = np.repeat(k, m)
    return x1, x2, 1.0 / (m * m)


def cell_centres(n):
    return nodes(n)[:2]


def isotropic(fun):
    """Kernel of (dx, dy) from a covariance of the distance."""
    return lambda dx, dy: fun(np.sqrt(dx * dx + dy * dy))


def nystrom(m, s, kernel):
    """Nystrom eigenpairs: B = sqrt(W) Sigma sqrt(W) (Sigma_kq = kernel(x_k - x_q)),
    all eigenpairs of B, the s largest in descending order; nodal
    eigenfunctions psi_j(x_q) = v_qj / sqrt(w) (so that sum_q w psi_i psi_j =
    delta_ij). Returns (theta (s,), psi (m*m, s), all eigenvalues descending)."""
    x1, x2, w = nodes(m)
    Sigma = kernel(x1[:, None] - x1[None, :], x2[:, None] - x2[None, :])
    B = w * Sigma
    ev, V = np.linalg.eigh(B)
    order = np.argsort(ev)[::-1]
    ev, V = ev[order], V[:, order]
    return ev[:s].copy(), V[:, :s] / np.sqrt(w), ev


def interpolate(n, m, theta, psi, kernel):
    """Nystrom interpolation formula at the n x n cell centres:
    psi_j(x) = 1/theta_j sum_q w C(x, x_q) psi_j(x_q); returns (n*n, s)."""
    y1, y2 = cell_centres(n)
    x1, x2, w = nodes(m)
    K = kernel(y1[:, None] - x1[None, :], y2[:, None] - x2[None, :])
    return (K @ (w * psi)) / theta[None, :]


def field(n, m, theta, psi, kernel, y):
    """k = exp(z), z = sum_j sqrt(theta_j) y_j psi_j at the n x n cell centres (eq. truncatedKL)."""
    P = interpolate(n, m, theta, psi, kernel)
    return np.exp(P @ (np.sqrt(theta) * np.asarray(y, dtype=np.float64)))
