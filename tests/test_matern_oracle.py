"""Pins of the Matern / Nystrom oracle (Sec. 5, eq. matern): closed forms
against the Bessel form, exact identities of the discrete eigenproblem, and
convergence to the separable kernel's closed-form eigenvalues."""
import numpy as np
import pytest

import oracle as O
from oracle import matern as MT


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_closed_forms_equal_the_bessel_form(nu):
    pytest.importorskip("scipy")
    r = np.array([0.0, 1e-3, 0.05, 0.2, 0.7, 1.4])
    a = MT.matern(r, nu, 0.3, sigma=1.3)
    b = MT.matern_bessel(r, nu, 0.3, sigma=1.3)
    assert np.allclose(a, b, rtol=1e-12, atol=0)


@pytest.mark.parametrize("nu", [1.0, 2.0])
def test_integer_order_against_the_integral_representation(nu):
    """K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt (an independent route to
    the Bessel function) in eq. matern, at several distances."""
    pytest.importorskip("scipy")
    from math import gamma
    from scipy.integrate import quad

    lam, sigma = 0.3, 1.1
    for r in [1e-3, 0.02, 0.3, 1.2]:
        z = np.sqrt(2 * nu) * r / lam
        t_max = np.log(400.0 / z) + 4.0  # exp(-z cosh t) below 1e-80 beyond it
        K = quad(lambda t: np.exp(-z * np.cosh(t)) * np.cosh(nu * t), 0, t_max, epsabs=0, epsrel=1e-13, limit=400)[0]
        want = sigma ** 2 * 2 ** (1 - nu) / gamma(nu) * z ** nu * K
        assert MT.matern(r, nu, lam, sigma) == pytest.approx(want, rel=1e-11)
    assert MT.matern(0.0, nu, lam, sigma) == sigma ** 2


def _kern(nu=1.5, lam=0.3, sigma=1.0):
    return MT.isotropic(lambda r: MT.matern(r, nu, lam, sigma))


def test_trace_identity_and_orthonormality():
    m, sigma = 12, 1.7
    theta, psi, ev = MT.nystrom(m, 20, _kern(sigma=sigma))
    # sum of all eigenvalues = trace(B) = sum_q w C(0) = sigma^2 (Sec. 6's identity, discrete)
    assert ev.sum() == pytest.approx(sigma ** 2, rel=1e-12)
    assert np.all(np.diff(theta) <= 0) and theta[-1] > 0
    w = 1.0 / m ** 2
    G = w * psi.T @ psi
    assert np.allclose(G, np.eye(20), atol=1e-12)


def test_interpolation_reproduces_the_nodal_values():
    # level cells = Nystrom nodes: the interpolation formula is the discrete eigen-equation
    m = 16
    k = _kern(nu=0.5, lam=0.2)
    theta, psi, _ = MT.nystrom(m, 30, k)
    P = MT.interpolate(m, m, theta, psi, k)
    assert np.allclose(P, psi, rtol=0, atol=1e-11 * np.abs(psi).max())


def test_separable_kernel_eigenvalues_converge_to_closed_form():
    """Same Nystrom machinery on the separable exponential kernel: its top
    eigenvalues approach the closed-form products theta_a theta_b (oracle
    or_modes) at the midpoint rule's second order."""
    lam = 0.3
    orc = O.Oracle(n_levels=2, n0=8, s=12, corr_len=lam, sampler="mc", seed=1, R=1)
    _, _, th_exact, _ = orc.modes()
    sep = lambda dx, dy: np.exp(-np.abs(dx) / lam - np.abs(dy) / lam)
    errs = []
    for m in (16, 32):
        theta, _, _ = MT.nystrom(m, 12, sep)
        errs.append(np.max(np.abs(theta - th_exact) / th_exact))
    assert errs[0] < 0.1 and errs[1] < errs[0] / 3.5  # h^2: 7.1 % then 1.7 %
