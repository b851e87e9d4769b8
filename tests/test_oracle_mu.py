"""Pins of the oracle's density <-> chemical-potential relation of the FD/BE
equilibrium (Sec. 4, g_nu before Eq. rho-fd-be-eq; Sec. 9.1, Eq.
rho-def-eq; the inverse of Sec. 9.1.2).  CPU only."""
import math

import numpy as np
import pytest

import oracle

THETA = 1.0 / 270.0


def test_fd_integral_closed_forms():
    """g_1(z) = ln(1 + z) (FD) and -ln(1 - z) (BE); at z = 1 the FD integral
    is the Dirichlet eta function, g_nu(1) = (1 - 2^{1-nu}) zeta(nu); for
    z -> 0 both tend to z -+ z^2 / 2^nu."""
    special = pytest.importorskip("scipy.special")
    for eta in (-20.0, -3.0, -0.5, 0.0, 0.7, 5.0, 40.0, 270.0):
        # ln(1 + e^eta), written without cancellation on either side
        closed = math.log1p(math.exp(eta)) if eta < 30 else eta + math.log1p(math.exp(-eta))
        assert abs(oracle.fd_integral(1.0, eta) / closed - 1) < 1e-13, eta
    for eta in (-20.0, -3.0, -0.5, -1e-3):
        assert abs(oracle.fd_integral(1.0, eta, "be") / (-math.log1p(-math.exp(eta))) - 1) < 1e-13, eta
    for nu in (0.5, 1.5, 2.0, 2.5):
        assert abs(oracle.fd_integral(nu, 0.0) / ((1 - 2 ** (1 - nu)) * special.zeta(nu)) - 1) < 1e-13, nu
    for nu in (0.5, 1.5):
        z = math.exp(-25.0)
        assert abs(oracle.fd_integral(nu, -25.0) / (z - z * z / 2 ** nu) - 1) < 1e-13
        assert abs(oracle.fd_integral(nu, -25.0, "be") / (z + z * z / 2 ** nu) - 1) < 1e-13


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_sommerfeld_expansion(nu):
    """Sec. 9.1, Eq. sommerfeld-approx-eq: for mu/theta >> 1
    g_nu = (mu/theta)^nu / Gamma(nu+1) [1 + nu(nu-1) pi^2/6 (theta/mu)^2
    + nu(nu-1)(nu-2)(nu-3) 7 pi^4/360 (theta/mu)^4 + ...]; at mu/theta = 270
    (copper, Sec. 9.1) the two printed corrections leave less than 1e-12,
    and the paper's 1e-8 with one of them."""
    eta = 270.0
    lead = eta ** nu / math.gamma(nu + 1)
    c1 = nu * (nu - 1) * math.pi ** 2 / 6 / eta ** 2
    c2 = nu * (nu - 1) * (nu - 2) * (nu - 3) * 7 * math.pi ** 4 / 360 / eta ** 4
    g = oracle.fd_integral(nu, eta)
    assert abs(g / (lead * (1 + c1 + c2)) - 1) < 1e-12
    assert abs(g / (lead * (1 + c1)) - 1) < 1e-8


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("stat,theta,mu", [("fd", THETA, 1.0), ("fd", 0.1, 1.0), ("fd", 0.3, -0.2), ("be", 0.5, -0.3)])
def test_density_is_the_weight_integral(D, stat, theta, mu):
    """Eq. rho-def-eq: rho = (pi theta)^{D/2} g_{D/2}(e^{mu/theta}) equals the
    zeroth weight integral I_0 of the same FD/BE distribution (Sec. 3, Eq.
    i2n-cont2, the radial integral of a different integrand)."""
    I0 = oracle.weight_integrals(D, stat, theta, mu, nmax=0)[0]
    rho = oracle.density_of_mu(D, theta, mu, stat)
    assert abs(rho / I0 - 1) < 1e-12, (rho, I0)


def test_printed_densities():
    """Sec. 9.4: at mu = 1 the steady densities are rho_2D = 3.142 and
    rho_3D = 4.189 (theta = 1/270)."""
    assert abs(oracle.density_of_mu(2, THETA, 1.0) - 3.142) < 5e-4
    assert abs(oracle.density_of_mu(3, THETA, 1.0) - 4.189) < 5e-4


def test_mu_of_density_inverse():
    """The inverse: in 2D in closed form, mu = theta ln(e^{rho/(pi theta)} - 1)
    (g_1 = ln(1 + z)); in 1D and 3D the round trip rho -> mu -> rho."""
    for rho in (0.05, 1.0, 3.0, 3.3):
        want = THETA * math.log(math.expm1(rho / (math.pi * THETA)))
        assert abs(oracle.mu_of_density(2, THETA, rho) - want) < 1e-12 * max(1.0, abs(want))
    for D in (1, 3):
        for theta in (THETA, 0.1):
            for rho in (1e-3, 0.3, 2.0, 4.5):
                mu = oracle.mu_of_density(D, theta, rho)
                assert abs(oracle.density_of_mu(D, theta, mu) / rho - 1) < 1e-13, (D, theta, rho)
    mu = oracle.mu_of_density(2, 0.5, 0.2, "be")
    assert mu < 0 and abs(oracle.density_of_mu(2, 0.5, mu, "be") / 0.2 - 1) < 1e-13
