"""Physics pins of the oracle's time step: conservation, shear-wave viscosity,
Poiseuille start-up and steady profiles, the isothermal Riemann plateau, the
Ohm's-law linearity, and a textbook D2Q9 BGK step in the Hermite limit.
CPU only."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1710_09472_gb300 import workloads as wl

THETA = 1.0 / 270.0


def test_mass_conserved_with_bounce_back():
    """Halfway bounce-back and BGK conserve sum rho to round-off (Sec. 9.1)."""
    shape = (24, 20)
    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.75, seed=7)
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=0.7, E=(2e-4, 1e-4), B=(0, 0, 1e-3), force="term")
    rho0 = 1.0 + 0.01 * wl.uniform01(9, mask.size).reshape(shape)
    f = m.init_equilibrium(shape, mask, rho0)
    _, _, t0 = m.moments(shape, mask, f)
    m.step(shape, mask, f, 200)
    _, _, t1 = m.moments(shape, mask, f)
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]


@pytest.mark.parametrize("force", ["term", "shift"])
def test_uniform_force_momentum_growth(force):
    """In a periodic box without walls, sum_x j grows by sum_x rho E per step."""
    shape = (6, 5, 4)
    E = (1e-4, -2e-4, 3e-5)
    m = oracle.Model("D3V19", "fd", THETA, 1.0, tau=0.8, E=E, force=force)
    rho0 = 1.0 + 0.02 * wl.uniform01(3, 120).reshape(shape)
    f = m.init_equilibrium(shape, None, rho0)
    _, _, t0 = m.moments(shape, None, f)
    m.step(shape, None, f, 7)
    _, _, t1 = m.moments(shape, None, f)
    for d in range(3):
        assert abs(t1[1 + d] - t0[1 + d] - 7 * t0[0] * E[d]) < 1e-13


def test_shear_wave_viscosity():
    """A shear wave u_x = U sin(k y) decays as exp(-nu k^2 t) with the lattice
    kinematic viscosity nu = (tau - 1/2)/3 (Sec. 9.3, eta = (tau - dt/2)/3)."""
    ny, tau = 64, 0.8
    shape = (ny, 1)
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=tau)
    k = 2 * math.pi / ny
    y = np.arange(ny)
    u = np.zeros((2,) + shape)
    u[0, :, 0] = 1e-4 * np.sin(k * y)
    f = m.init_equilibrium(shape, None, np.ones(shape), u)
    amps = []
    t_marks = [100, 600]
    done = 0
    for t in t_marks:
        m.step(shape, None, f, t - done)
        done = t
        rho, j, _ = m.moments(shape, None, f)
        ux = j[0, :, 0] / rho[:, 0]
        amps.append(2.0 / ny * np.sum(ux * np.sin(k * y)))
    nu_meas = math.log(amps[0] / amps[1]) / (k * k * (t_marks[1] - t_marks[0]))
    nu = (tau - 0.5) / 3.0
    assert abs(nu_meas / nu - 1) < 3e-3, nu_meas


def _poiseuille_series(y, t, a, nu, y0, H, nterms=400):
    s = y - y0
    u = a / (2 * nu) * s * (H - s)
    for n in range(1, 2 * nterms, 2):
        u -= 4 * a * H * H / (nu * math.pi ** 3 * n ** 3) * np.sin(n * math.pi * s / H) * math.exp(
            -nu * n * n * math.pi ** 2 * t / (H * H))
    return u


@pytest.mark.parametrize("force", ["shift", "term"])
def test_poiseuille_startup_32x64(force):
    """Channel of 64 rows with solid rows y = 0, 63 (halfway walls at y = 0.5 and
    62.5, H = 62), E_x = 1e-6, tau = 0.8, 5000 steps: the profile follows the
    analytic start-up series of du/dt = a + nu u'' (Sec. 9.3, Eq.
    poiseuille-ux-eq in its time-dependent form); x is periodic, so two columns
    suffice."""
    w = wl.poiseuille_32x64()
    shape = (64, 2)
    solid = wl.channel_mask(shape)
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=w["tau"], E=w["E"], force=force)
    f = m.init_equilibrium(shape, solid, np.ones(shape))
    m.step(shape, solid, f, w["steps"])
    rho, j, _ = m.moments(shape, solid, f)
    ux = j[0, 1:-1, 0] / rho[1:-1, 0]
    y = np.arange(1, 63, dtype=np.float64)
    nu = (w["tau"] - 0.5) / 3.0
    ref = _poiseuille_series(y, w["steps"], w["E"][0], nu, 0.5, 62.0)
    err = np.max(np.abs(ux - ref)) / np.max(ref)
    assert err < 5e-3, err


@pytest.mark.slow
def test_poiseuille_steady_parabola():
    """Long run: the steady profile is a parabola of curvature -a/nu."""
    shape = (64, 1)
    solid = wl.channel_mask(shape)
    tau, a = 0.8, 1e-6
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=tau, E=(a, 0.0), force="shift")
    f = m.init_equilibrium(shape, solid, np.ones(shape))
    m.step(shape, solid, f, 80000)
    rho, j, _ = m.moments(shape, solid, f)
    ux = j[0, 1:-1, 0] / rho[1:-1, 0]
    y = np.arange(1, 63, dtype=np.float64)
    p = np.polyfit(y, ux, 2)
    nu = (tau - 0.5) / 3.0
    assert abs(2 * p[0] / (-a / nu) - 1) < 1e-3
    resid = ux - np.polyval(p, y)
    assert np.max(np.abs(resid)) < 1e-4 * np.max(ux)


def _riemann_star(rho_l, rho_r):
    """Isothermal Riemann problem (gas at rest on both sides): rarefaction to the
    left, shock to the right; u* = c ln(rho_l/rho*) = c (rho* - rho_r)/sqrt(rho* rho_r)."""
    g = lambda r: math.log(rho_l / r) - (r - rho_r) / math.sqrt(r * rho_r)
    return brentq(g, rho_r, rho_l, xtol=1e-15)


def test_riemann_plateau():
    """Shock tube rho_L = 1.05 | rho_R = 1.0, tau = 0.6, 2000 steps on 4096 cells with
    closed ends: the plateau between rarefaction and shock has the isothermal
    exact density rho* and velocity u* with sound speed c^2 = thetabar in xi
    units (pressure rho thetabar, Sec. 6) (Sec. 9.2 compares with the classical
    solution scaled by sqrt(thetabar))."""
    w = wl.riemann_4096x8()
    shape = (1, 4096)
    solid = wl.end_walls_mask(shape)
    rho_init = wl.riemann_density(shape, 1.05, 1.0, 2048)
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=w["tau"])
    f = m.init_equilibrium(shape, solid, rho_init)
    m.step(shape, solid, f, w["steps"])
    rho, j, _ = m.moments(shape, solid, f)
    rs = _riemann_star(1.05, 1.0)
    c = math.sqrt(m.const["thetabar"])
    us = c * math.log(1.05 / rs)
    # plateau: between the rarefaction tail and the shock; sample around the split
    cl = c * m.const["cs"]  # lattice-unit sound speed
    xs = 2048
    plateau = slice(xs - 100, xs + 300)
    r_pl = rho[0, plateau]
    u_pl = j[0, 0, plateau] / r_pl
    assert abs(np.median(r_pl) - rs) < 2e-4, (np.median(r_pl), rs)
    assert abs(np.median(u_pl) / us - 1) < 5e-3, (np.median(u_pl), us)
    # the shock moves at s = c sqrt(rho*/rho_R) (lattice units)
    s_lat = cl * math.sqrt(rs / 1.0)
    x_shock = xs + s_lat * w["steps"]
    mid = 0.5 * (rs + 1.0)
    idx = np.where(rho[0, xs:4095] < mid)[0][0] + xs
    assert abs(idx - x_shock) < 15, (idx, x_shock)


def test_ohm_linearity_2d():
    """Sec. 9.4: the mean x-velocity through a random porous medium is linear in
    E.  Two fields a factor 2 apart give <u_x>/E equal to 1e-4 (the nonlinearity
    is O(u^2))."""
    shape = (40, 40)
    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.8, seed=11)
    ratios = []
    for E in (1e-6, 2e-6):
        m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=0.9, E=(E, 0.0), force="shift")
        f = m.init_equilibrium(shape, mask, np.ones(shape))
        m.step(shape, mask, f, 3000)
        rho, j, tot = m.moments(shape, mask, f)
        fluid = mask == 0
        ratios.append(np.mean(j[0][fluid] / rho[fluid]) / E)
    assert abs(ratios[1] / ratios[0] - 1) < 1e-4, ratios


def _textbook_d2q9_step(f, solid, tau, shape):
    """Textbook D2Q9 BGK with halfway bounce-back, written independently
    (standard velocity set and weights 4/9, 1/9, 1/36; equilibrium
    rho w (1 + 3 e.v + 4.5 (e.v)^2 - 1.5 v^2))."""
    e = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    opp = [0, 2, 1, 4, 3, 6, 5, 8, 7]
    rho = f.sum(axis=0)
    v = np.einsum("a...,ad->d...", f, e.astype(float)) / np.where(rho == 0, 1, rho)
    ev = np.einsum("ad,d...->a...", e.astype(float), v)
    feq = rho * w[:, None, None] * (1 + 3 * ev + 4.5 * ev ** 2 - 1.5 * (v ** 2).sum(axis=0))
    fs = f - (f - feq) / tau
    fs[:, solid == 1] = 0
    out = np.zeros_like(f)
    for a in range(9):
        pulled = np.roll(fs[a], shift=(e[a][1], e[a][0]), axis=(0, 1))
        src_solid = np.roll(solid, shift=(e[a][1], e[a][0]), axis=(0, 1)) == 1
        out[a] = np.where(src_solid, fs[opp[a]], pulled)
    out[:, solid == 1] = 0
    return out


def test_hermite_limit_step_is_textbook():
    """With the Hermite weight the whole step (collision, streaming and
    bounce-back) equals a textbook D2Q9 BGK step."""
    shape = (12, 16)
    mask, _ = wl.boolean_obstacles(shape, 2.0, 0.8, seed=5)
    m = oracle.Model("D2V9", "mb", 1.0, 0.0, tau=0.75)
    assert np.all(m.e[:, :2] == np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1],
                                          [-1, 1]]))
    rho = 1.0 + 0.05 * wl.uniform01(4, mask.size).reshape(shape)
    u = 0.02 * (wl.uniform01(5, 2 * mask.size).reshape((2,) + shape) - 0.5)
    f = m.init_equilibrium(shape, mask, rho, u)
    g = f.reshape(9, *shape).copy()
    for _ in range(5):
        m.step(shape, mask, f, 1)
        g = _textbook_d2q9_step(g, mask, 0.75, shape)
        assert np.max(np.abs(f.reshape(9, *shape) - g)) < 1e-14
