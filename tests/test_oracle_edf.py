"""Pins of the oracle's equilibrium, forcing term and collision: moment
identities that the paper derives, the equality of its two printed EDF forms,
and the textbook Hermite limit.  CPU only."""
import numpy as np
import pytest

import oracle

THETA = 1.0 / 270.0


def _rng():
    return np.random.default_rng(12345)


def _moments(m, f):
    rho = f.sum()
    j = (f[:, None] * m.xi).sum(axis=0)
    P = np.einsum("a,ai,aj->ij", f, m.xi, m.xi)
    return rho, j, P


@pytest.mark.parametrize("vel", ["D1V3", "D2V9", "D3V19", "D3V27"])
def test_equilibrium_moments(vel):
    """sum f^eq = rho, sum f^eq xi = rho u, sum f^eq xi xi = rho (thetabar delta + u u)
    (Sec. 2 Eqs. rho-def-eq, vel-def-eq, theta-bar-def-eq; Sec. 6 pi_ij)."""
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=0.8)
    D = m.D
    r = _rng()
    for _ in range(20):
        rho = 0.5 + r.random()
        u = np.zeros(3)
        u[:D] = r.normal(size=D) * 0.05
        f = m.equilibrium(rho, u[:D])
        R, j, P = _moments(m, f)
        assert abs(R - rho) < 1e-14 * rho
        assert np.max(np.abs(j - rho * u)) < 1e-15
        expect = rho * (m.const["thetabar"] * np.eye(3) + np.outer(u, u))
        expect[D:, :] = 0
        expect[:, D:] = 0
        assert np.max(np.abs(P - expect)) < 1e-14


@pytest.mark.parametrize("vel", ["D1V3", "D2V9", "D3V19", "D3V27"])
def test_equilibrium_printed_forms_agree(vel):
    """The reduced EDF the paper simulates (Sec. 9.1) equals the full second-order
    EDF (Sec. 4, Eq. edf-second-order-exp-eq, discrete) with thetabar = I2/I0, and
    the direct N=2 derivation of Sec. 5.1 (Eq. feq-reduce-general-method-...)."""
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=0.8)
    c = m.const
    D = m.D
    c0, c1, c2, cb, cp, th = c["c0"], c["c1"], c["c2"], c["cbar2"], c["cprime2"], c["thetabar"]
    I0, I2, I4, Dl = c["I0"], c["I2"], c["I4"], c["Delta2"]
    r = _rng()
    for _ in range(10):
        rho = 0.7 + r.random()
        u = r.normal(size=D) * 0.03
        got = m.equilibrium(rho, u)
        full = np.zeros(m.Q)
        direct = np.zeros(m.Q)
        u2 = u @ u
        for a in range(m.Q):
            xi = m.xi[a, :D]
            xu, x2 = xi @ u, xi @ xi
            full[a] = rho * m.w[a] * (c0 ** 2 + c1 ** 2 * xu + 0.5 * c2 * (c2 * th + cp) * x2
                                      + 0.5 * c2 ** 2 * xu ** 2 + 0.5 * c2 * cb * (D * th + u2) * x2
                                      + 0.5 * (cb * x2 + cp) * (D * (c2 * th + cp) + c2 * u2 + D * cb * (D * th + u2)))
            direct[a] = rho / I0 * m.w[a] * (1 + I0 / I2 * xu + I0 / I4 * 0.5 * xu ** 2
                                             + 0.5 * u2 * (I0 / I4 * (Dl ** 2 - 1) / D * x2 - I2 / I4 * Dl ** 2))
        assert np.max(np.abs(got - full)) < 1e-14
        assert np.max(np.abs(got - direct)) < 1e-14


def test_hermite_limit_is_textbook_bgk():
    """With the Hermite weight (MB, theta = 1; I_2N = 1) the EDF is the textbook
    D2Q9 equilibrium rho w (1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2), v = c_s u the
    lattice-unit velocity (Sec. 3: c_K = 1, cbar_K = 0, c'_K = -1)."""
    m = oracle.Model("D2V9", "mb", 1.0, 0.0, tau=0.8)
    assert abs(m.const["cs"] - 1 / np.sqrt(3)) < 1e-14
    r = _rng()
    for _ in range(10):
        rho = 0.8 + 0.4 * r.random()
        v = r.normal(size=2) * 0.05  # lattice units
        u = v / m.const["cs"]
        f = m.equilibrium(rho, u)
        ev = m.e[:, :2] @ v
        textbook = rho * m.w * (1 + 3 * ev + 4.5 * ev ** 2 - 1.5 * (v @ v))
        assert np.max(np.abs(f - textbook)) < 1e-14


@pytest.mark.parametrize("vel", ["D1V3", "D2V9", "D3V19", "D3V27"])
def test_force_term_moments(vel):
    """Sec. 7: the explicit term conserves mass and injects momentum rho a;
    for the magnetic part rho (u x B) via the identity J2 Delta2^2 -
    (D+2)(Delta2^2 - 1)/D = 1 (Eq. force-eq1, force-eq2).  In 1D only E_x acts."""
    B = {"D1V3": (0.0, 0.0, 0.0), "D2V9": (0.0, 0.0, 3e-3)}.get(vel, (1e-3, -2e-3, 3e-3))
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=0.8, B=B)
    D = m.D
    r = _rng()
    for _ in range(10):
        rho = 0.8 + 0.4 * r.random()
        u = np.zeros(3)
        u[:D] = r.normal(size=D) * 0.02
        E = np.zeros(3)
        E[:D] = r.normal(size=D) * 1e-3
        S = m.force_term(rho, u[:D], E[:D])
        assert abs(S.sum()) < 1e-16
        mom = (S[:, None] * m.xi).sum(axis=0)
        expect = rho * (E + np.cross(u, m.B))
        assert np.max(np.abs(mom - expect)) < 1e-16, (mom, expect)


@pytest.mark.parametrize("force", ["shift", "term"])
def test_collision_conserves_and_forces(force):
    """A collision conserves mass exactly and changes the momentum by
    rho (E + u x B) per step in both force modes (Sec. 7)."""
    B = (0.0, 0.0, 2e-3)
    E = (3e-4, -1e-4)
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=0.7, E=E, B=B, force=force)
    r = _rng()
    for _ in range(10):
        rho = 0.8 + 0.4 * r.random()
        u = r.normal(size=2) * 0.02
        f = m.equilibrium(rho, u) * (1 + 0.01 * r.normal(size=m.Q))
        R, j, _ = _moments(m, f)
        fo = m.collide_cell(f)
        R2, j2, _ = _moments(m, fo)
        assert abs(R2 - R) < 1e-15
        uu = np.zeros(3)
        uu[:2] = j[:2] / R
        dj = R * (np.array([E[0], E[1], 0.0]) + np.cross(uu, np.array(B)))
        assert np.max(np.abs(j2 - j - dj)) < 2e-16


def test_equilibrium_is_fixed_point_without_force():
    """Without force, f^eq is left unchanged by the collision."""
    m = oracle.Model("D3V19", "fd", THETA, 1.0, tau=0.8)
    f = m.equilibrium(1.1, np.array([0.01, -0.02, 0.005]))
    assert np.max(np.abs(m.collide_cell(f) - f)) < 1e-15
