"""Pins of the oracle's local-chemical-potential model: the second-order EDF
of Sec. 9.1, Eq. feq-exp-2nd-order-eq, with each cell's reduced temperature
thetabar = I_2/I_0 taken at its own chemical potential (the weight-equals-EDF
choice of Sec. 5, Eq. omega-feq, with the lattice of the fixed weight) instead
of the constant-thetabar approximation of Sec. 9.1.  CPU only."""
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1710)


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
@pytest.mark.parametrize("stat,theta,mu", [("fd", 1.0 / 270.0, 1.0), ("fd", 0.1, 1.0), ("be", 0.5, -0.3),
                                           ("mb", 1.0, 0.0)])
def test_full_edf_at_weight_thetabar_is_the_simulated_edf(vel, stat, theta, mu):
    """With thetabar = I_2/I_0 of the weight, Eq. feq-exp-2nd-order-eq equals
    the simulated Eq. feq-reduced-applied-electrons-in-metals-eq (the Sec. 9.1
    identity c2 thetabar + c'2 + D cbar2 thetabar = 0)."""
    m = oracle.Model(vel, stat, theta, mu)
    for _ in range(5):
        u = 0.05 * RNG.standard_normal(m.D)
        rho = m.const["I0"] * (1 + 0.1 * RNG.standard_normal())
        a = m.equilibrium(rho, u)
        b = m.equilibrium_thetabar(rho, u, m.const["thetabar"])
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
def test_full_edf_moments_carry_the_local_thetabar(vel):
    """For any thetabar the discrete EDF has sum f = rho, sum f xi = rho u and
    sum f xi_i xi_j = rho (thetabar delta_ij + u_i u_j): the lattice
    quadrature is exact for the products of the polynomials up to N = 2."""
    m = oracle.Model(vel, "fd", 0.1, 1.0)
    for _ in range(6):
        u = 0.05 * RNG.standard_normal(m.D)
        rho = m.const["I0"] * (1 + 0.2 * RNG.random())
        thb = m.const["thetabar"] * (0.5 + RNG.random())
        f = m.equilibrium_thetabar(rho, u, thb)
        xi = m.xi[:, : m.D]
        assert abs(f.sum() / rho - 1) < 1e-13
        np.testing.assert_allclose(f @ xi, rho * u, rtol=0, atol=1e-13 * rho)
        P = np.einsum("a,ai,aj->ij", f, xi, xi)
        np.testing.assert_allclose(P, rho * (thb * np.eye(m.D) + np.outer(u, u)), rtol=0, atol=1e-12 * rho)


@pytest.mark.parametrize("stat,mu", [("fd", 1.0), ("fd", -0.2), ("be", -0.3)])
def test_thetabar_2d_closed_form_equals_weight_integrals(stat, mu):
    """D = 2: the closed form (g_1 = ln(1+z), g_2 = -Li_2(-z) for FD; the BE
    analogues) equals mu_of_density followed by I_2/I_0 from the adaptive
    quadrature of the weight integrals, two independent routes."""
    theta = 0.1
    I0w = oracle.density_of_mu(2, theta, mu, stat)
    for r in (0.3, 0.8, 1.0, 1.25, 2.0):
        mu_c = oracle.mu_of_density(2, theta, r * I0w, stat)
        slow = oracle.thetabar_of_mu(2, theta, mu_c, stat)
        fast = oracle.thetabar_of_density(2, stat, theta, mu, np.array([r * I0w]))[0]
        assert abs(fast / slow - 1) < 1e-12, (stat, mu, r, fast, slow)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_thetabar_limits(D):
    """Degenerate limit (Sec. 9.1, Eq. sommerfeld-approx-eq): with
    g_nu = eta^nu / Gamma(nu+1) [1 + nu (nu-1) pi^2 / (6 eta^2) + ...] the ratio
    thetabar = theta g_{D/2+1} / (2 g_{D/2}) is mu / (D+2) [1 + D pi^2 / (6 eta^2)]
    up to O(eta^-4); classical limit of the FD weight (exponent xi^2/theta,
    Eq. fd-dist-non-dim-eq) thetabar -> theta/2; the MB weight of the
    classical LBM has thetabar = theta at any mu (Sec. 9.1)."""
    theta, mu = 1.0 / 270.0, 1.0
    eta = mu / theta
    thb = oracle.thetabar_of_mu(D, theta, mu, "fd")
    assert abs(thb / (mu / (D + 2) * (1 + D * math.pi ** 2 / (6 * eta ** 2))) - 1) < 1e-8
    theta = 0.2
    thb = oracle.thetabar_of_mu(D, theta, -25 * theta, "fd")
    assert abs(thb / (theta / 2) - 1) < 1e-9
    assert abs(oracle.thetabar_of_mu(D, theta, 0.3, "mb") / theta - 1) < 1e-12


def test_thetabar_3d_route():
    """D = 3 (no closed form): the cell-by-cell route, on a density from the
    Sommerfeld side where the two printed corrections of Eq.
    sommerfeld-approx-eq fix rho(mu) and thetabar(mu) to 1e-10."""
    theta = 1.0 / 270.0
    nu = 1.5
    for mu in (0.8, 1.0, 1.3):
        eta = mu / theta

        def g(n):
            return eta ** n / math.gamma(n + 1) * (1 + n * (n - 1) * math.pi ** 2 / 6 / eta ** 2
                                                    + n * (n - 1) * (n - 2) * (n - 3) * 7 * math.pi ** 4 / 360 / eta ** 4)

        rho = (math.pi * theta) ** nu * g(nu)
        want = theta * g(nu + 1) / (2 * g(nu))
        got = oracle.thetabar_of_density(3, "fd", theta, 1.0, np.array([rho]))[0]
        assert abs(got / want - 1) < 1e-10, (mu, got, want)


def test_local_model_mb_is_the_base_model():
    """With the MB weight thetabar does not depend on mu, so the local model
    is the simulated model (up to the rounding of the two EDF forms)."""
    m = oracle.Model("D2V9", "mb", 1.0, 0.0, tau=0.8, E=(1e-4, 0.0), B=(0.0, 0.0, 1e-2))
    shape = (12, 20)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[5:7, 8:11] = 1
    rho = m.const["I0"] * (1 + 0.02 * RNG.standard_normal(shape))
    f0 = m.init_equilibrium(shape, solid, rho)
    a = m.step(shape, solid, f0.copy(), 30)
    b = m.step_local_mu(shape, solid, f0.copy(), 30)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def _wave_speed(m, nx, steps, amp, local):
    """Speed of a standing density wave of wavelength nx in a periodic row
    (D2V9, one cell high): the zero crossings of j_x at x = nx/4."""
    shape = (1, nx)
    x = np.arange(nx)
    rho0 = m.const["I0"]
    f = m.init_equilibrium(shape, None, (rho0 * (1 + amp * np.cos(2 * np.pi * x / nx)))[None, :])
    probe = []
    for _ in range(steps):
        if local:
            m.step_local_mu(shape, None, f, 1)
        else:
            m.step(shape, None, f, 1)
        probe.append(m.moments(shape, None, f)[1][0, 0, nx // 4])
    probe = np.array(probe)
    s = np.sign(probe)
    cross = np.flatnonzero(s[1:] != s[:-1])
    tc = np.array([c + probe[c] / (probe[c] - probe[c + 1]) for c in cross])
    period = 2 * float(np.mean(np.diff(tc)))
    return nx / period


def test_local_model_sound_speed_is_the_fermi_gas_one():
    """The local model has the FD equation of state p = rho thetabar(rho): its
    sound speed in lattice units is c_s sqrt(d(rho thetabar)/d rho) =
    c_s sqrt(thetabar + rho thetabar'(rho)) (in the degenerate 2D limit
    sqrt(2) times the constant-thetabar model's c_s sqrt(thetabar)).  Both are
    measured from standing waves (FD, theta = 0.1, mu = 1, tau = 0.6)."""
    m = oracle.Model("D2V9", "fd", 0.1, 1.0, tau=0.6)
    rho0, cs, thw = m.const["I0"], m.const["cs"], m.const["thetabar"]
    h = 1e-5 * rho0
    dth = (m.local_thetabar(np.array([rho0 + h]))[0] - m.local_thetabar(np.array([rho0 - h]))[0]) / (2 * h)
    want_local = cs * math.sqrt(thw + rho0 * dth)
    want_fixed = cs * math.sqrt(thw)
    nx = 64
    c_local = _wave_speed(m, nx, 600, 1e-5, True)
    c_fixed = _wave_speed(m, nx, 600, 1e-5, False)
    print(f"sound speed: local {c_local:.6f} (want {want_local:.6f}), fixed {c_fixed:.6f} (want {want_fixed:.6f})")
    assert abs(c_fixed / want_fixed - 1) < 2e-3
    assert abs(c_local / want_local - 1) < 2e-3
    assert c_local / c_fixed > 1.2


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
def test_local_term_has_shell_constants(vel):
    """The CUDA collision adds rho w_a K_a (thetabar - thetabar_w) with
    K_a = 1/2 (c2 + D cbar2) [(c2 + D cbar2) xi_a^2 + D c'2], one constant per
    shell |e_a|^2, and relies on sum_a w_a K_a = 0 (the rest population's share
    then follows from the mass closure).  Both against the oracle's full EDF."""
    m = oracle.Model(vel, "fd", 0.1, 1.0)
    c = m.const
    g = c["c2"] + m.D * c["cbar2"]
    xi2 = np.sum(m.xi ** 2, axis=1)
    K = 0.5 * g * (g * xi2 + m.D * c["cprime2"])
    assert abs(np.sum(m.w * K)) < 1e-12 * np.sum(m.w * np.abs(K))
    for _ in range(4):
        u = 0.05 * RNG.standard_normal(m.D)
        rho = c["I0"] * (1 + 0.1 * RNG.random())
        d = c["thetabar"] * (RNG.random() - 0.5)
        diff = m.equilibrium_thetabar(rho, u, c["thetabar"] + d) - m.equilibrium(rho, u)
        np.testing.assert_allclose(diff, rho * m.w * K * d, rtol=0, atol=1e-12 * rho)


def _local_loss(m, shape, mask, f0, Efield, T, t_begin, wr, wj):
    f = f0.copy()
    L = 0.0
    for t in range(1, T + 1):
        m.step_local_mu(shape, mask, f, 1, Efield, rho_ref=1.0)
        if t > t_begin:
            rho, j, _ = m.moments(shape, mask, f)
            L += np.sum(wr * rho) + np.sum(wj * j)
    return L


@pytest.mark.parametrize("force", ["term", "shift"])
def test_local_mu_adjoint_vs_finite_differences(force):
    """The reverse sweep of the local model (Model.adjoint_local_mu) against
    central differences of its forward run (Model.step_local_mu): per-cell
    dL/dE, dL/dB_z, dL/dtau and dL/df_0 along a random direction (D2V9, FD
    theta = 0.5, mu = 0, 2% density noise, an obstacle)."""
    from paper_1710_09472_gb300 import workloads as wl

    shape = (10, 12)
    mask, _ = wl.boolean_obstacles(shape, 2.0, 0.8, seed=21)
    N = mask.size
    B = (0.0, 0.0, 2e-2)
    Efield = np.zeros((2,) + shape)
    Efield[0] = 1e-3 + 2e-4 * wl.normal(31, N).reshape(shape)
    Efield[1] = 3e-4 * wl.normal(32, N).reshape(shape)
    rho0 = 1.0 + 0.02 * wl.uniform01(33, N).reshape(shape)
    u0 = 0.01 * wl.normal(34, 2 * N).reshape((2,) + shape)
    wr = wl.normal(35, N).reshape(shape)
    wj = wl.normal(36, 2 * N).reshape((2,) + shape)
    tau, T, t_begin = 0.75, 10, 5

    def model(tau_=tau, B_=B):
        return oracle.Model("D2V9", "fd", 0.5, 0.0, tau=tau_, B=B_, force=force)

    m = model()
    f0 = m.init_equilibrium(shape, mask, rho0, u0)
    states = np.empty((T + 1, f0.size))
    states[0] = f0
    f = f0.copy()
    for t in range(T):
        m.step_local_mu(shape, mask, f, 1, Efield, rho_ref=1.0)
        states[t + 1] = f
    res = m.adjoint_local_mu(shape, mask, states, t_begin, T, wr, wj, Efield, rho_ref=1.0)
    L0 = _local_loss(m, shape, mask, f0, Efield, T, t_begin, wr, wj)
    assert abs(res["loss"] - L0) < 1e-12 * max(1, abs(L0))
    base = m.adjoint(shape, mask, states, t_begin, T, wr, wj, Efield)
    assert abs(base["gtau"] - res["gtau"]) > 1e-3 * abs(res["gtau"])  # the local terms matter

    fluid = np.argwhere(mask == 0)
    rng = np.random.default_rng(0)
    h = 1e-6
    for k in rng.choice(len(fluid), 3, replace=False):
        cell = tuple(fluid[k])
        for d in range(2):
            Ep, Em = Efield.copy(), Efield.copy()
            Ep[(d,) + cell] += h
            Em[(d,) + cell] -= h
            fd = (_local_loss(m, shape, mask, f0, Ep, T, t_begin, wr, wj)
                  - _local_loss(m, shape, mask, f0, Em, T, t_begin, wr, wj)) / (2 * h)
            assert abs(res["gE"][(d,) + cell] - fd) < 1e-6 * max(abs(fd), 1e-3), (cell, d)
    fd = (_local_loss(model(B_=(0.0, 0.0, B[2] + h)), shape, mask, f0, Efield, T, t_begin, wr, wj)
          - _local_loss(model(B_=(0.0, 0.0, B[2] - h)), shape, mask, f0, Efield, T, t_begin, wr, wj)) / (2 * h)
    assert abs(res["gB"][2] - fd) < 1e-6 * max(abs(fd), 1e-3), (res["gB"][2], fd)
    fd = (_local_loss(model(tau_=tau + h), shape, mask, f0, Efield, T, t_begin, wr, wj)
          - _local_loss(model(tau_=tau - h), shape, mask, f0, Efield, T, t_begin, wr, wj)) / (2 * h)
    assert abs(res["gtau"] - fd) < 1e-6 * max(abs(fd), 1e-3), (res["gtau"], fd)
    v = rng.normal(size=f0.size)
    v.reshape(m.Q, -1)[:, mask.reshape(-1) == 1] = 0.0
    fd = (_local_loss(m, shape, mask, f0 + h * v, Efield, T, t_begin, wr, wj)
          - _local_loss(m, shape, mask, f0 - h * v, Efield, T, t_begin, wr, wj)) / (2 * h)
    assert abs(float(res["lam0"] @ v) - fd) < 1e-7 * max(abs(fd), 1.0), (float(res["lam0"] @ v), fd)
