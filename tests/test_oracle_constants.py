"""Pins of the oracle's host-side constants (weight integrals, polynomial
coefficients, lattices) against values the paper prints and against closed
forms.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.conftest import load_golden

THETA = 1.0 / 270.0
MU = 1.0


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("D,vel,fname", [(2, "D2V9", "constants_2d.txt"), (3, "D3V19", "constants_3d.txt")])
def test_printed_tables(D, vel, fname):
    """Sec. 9.1.1 / 9.1.2 print c0..c'2, thetabar, w and c_s to 24 digits."""
    g = load_golden(fname)
    m = oracle.Model(vel, "fd", THETA, MU, tau=0.8)
    c = m.const
    for k in ["c0", "c1", "c2", "cbar2", "cprime2", "thetabar", "cs"]:
        assert rel(c[k], g[k]) < 2e-14, (k, c[k], g[k])
    assert rel(m.w[0], g["w0"]) < 2e-14
    n_s = 2 * D  # the axis vectors come first after the rest vector
    for a in range(1, n_s + 1):
        assert rel(m.w[a], g["ws"]) < 2e-14
    for a in range(n_s + 1, m.Q):
        assert rel(m.w[a], g["wl"]) < 2e-14


def _g_int(n, eta):
    """Complete Fermi-Dirac integral g_n(e^eta) of integer order n for large
    eta: the Sommerfeld series terminates, up to O(e^-eta) (Sec. 9.1, Eq.
    sommerfeld-approx-eq; g_n = sum_k 2(1-2^{1-2k}) zeta(2k) eta^{n-2k}/(n-2k)!)."""
    zeta = {0: -0.5, 1: math.pi ** 2 / 6, 2: math.pi ** 4 / 90, 3: math.pi ** 6 / 945}
    s = 0.0
    for k in range(0, n // 2 + 1):
        coef = 2.0 * (1.0 - 2.0 ** (1 - 2 * k)) * zeta[k]
        s += coef * eta ** (n - 2 * k) / math.factorial(n - 2 * k)
    if n == 1:  # g_1 = ln(1+e^eta) exactly
        s = eta + math.log1p(math.exp(-eta))
    return s


def test_fd_2d_integrals_closed_form():
    """In 2D, I_2N = pi theta^{N+1} g_{N+1}(z) / 2^N (substitute x = xi^2/theta
    in Eq. i2n-cont2); for integer order the Sommerfeld series is exact up to
    e^{-270}.  In particular I_0 = pi mu, rho_2D = pi at mu = 1 (Sec. 9.1.1, 9.4)."""
    I = oracle.weight_integrals(2, "fd", THETA, MU, nmax=4)
    eta = MU / THETA
    for N in range(5):
        closed = math.pi * THETA ** (N + 1) * _g_int(N + 1, eta) / 2 ** N
        assert rel(I[N], closed) < 1e-13, (N, I[N], closed)
    assert rel(I[0], math.pi) < 1e-15


def test_fd_3d_density():
    """Sec. 9.4 quotes rho_3D = 4.189 at mu = 1 (the sphere volume 4 pi/3 up to
    O(theta^2)); I_0 is that density for the normalised EDF."""
    I = oracle.weight_integrals(3, "fd", THETA, MU, nmax=2)
    assert abs(I[0] - 4.189) < 5e-4
    sommerfeld = 4 * math.pi / 3 * (1 + (math.pi ** 2 / 8) * THETA ** 2)
    assert rel(I[0], sommerfeld) < 1e-8  # Sec. 9.1.2: Sommerfeld good to ~1e-8


def test_mb_integrals_closed_form():
    """MB weight (2 pi theta)^{-D/2} exp(-xi^2/2 theta): I_2N = theta^N; theta = 1
    is the Hermite weight with I_2N = 1 (Sec. 3, Eq. i2n-hermite)."""
    for D in (1, 2, 3):
        for th in (1.0, 0.37):
            I = oracle.weight_integrals(D, "mb", th, 0.0, nmax=4)
            for N in range(5):
                assert rel(I[N], th ** N) < 1e-13, (D, th, N, I[N])


def test_be_2d_integral_closed_form():
    """BE weight in 2D: I_0 = -pi theta ln(1 - e^{mu/theta}) and
    I_2 = pi theta^2 Li_2(e^{mu/theta}) / 2 (mu < 0)."""
    from scipy.special import spence

    th, mu = 0.5, -0.3
    I = oracle.weight_integrals(2, "be", th, mu, nmax=1)
    z = math.exp(mu / th)
    assert rel(I[0], -math.pi * th * math.log1p(-z)) < 1e-13
    li2 = spence(1.0 - z)
    assert rel(I[1], math.pi * th ** 2 * li2 / 2) < 1e-12


def test_hermite_limit_lattices():
    """Sec. 8: with I_2N = 1 the lattices become the textbook ones."""
    I = np.ones(5)
    e, w, opp, cs = oracle.lattice("D2V9", I)
    assert abs(cs - 1 / math.sqrt(3)) < 1e-15
    assert np.allclose(sorted(w), sorted([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4), atol=1e-15)
    e, w, opp, cs = oracle.lattice("D1V3", I)
    assert np.allclose(sorted(w), sorted([2 / 3, 1 / 6, 1 / 6]), atol=1e-15)
    e, w, opp, cs = oracle.lattice("D3V15", I)
    assert np.allclose(sorted(w), sorted([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8), atol=1e-15)
    e, w, opp, cs = oracle.lattice("D3V19", I)
    assert np.allclose(sorted(w), sorted([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12), atol=1e-15)
    e, w, opp, cs = oracle.lattice("D3V27", I)
    assert np.allclose(sorted(w), sorted([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8), atol=1e-15)


def _delta_tensor_value(idx):
    """delta_{i1..iM}: the sum over all pairings of products of Kronecker deltas."""
    idx = list(idx)
    if not idx:
        return 1
    if len(idx) % 2:
        return 0
    first, rest = idx[0], idx[1:]
    tot = 0
    for k in range(len(rest)):
        if rest[k] == first:
            tot += _delta_tensor_value(rest[:k] + rest[k + 1:])
    return tot


@pytest.mark.parametrize("vel,D", [("D1V3", 1), ("D2V9", 2), ("D3V19", 3), ("D3V27", 3)])
def test_quadrature_moments_bruteforce(vel, D):
    """Sec. 8, Eq. quadrature-eq-2: sum_a w_a e_a^{i1}..e_a^{iM} = I_M c_s^M delta_{i1..iM}
    for every index tuple with M <= 5 (odd orders vanish)."""
    I = oracle.weight_integrals(D, "fd", THETA, MU, nmax=4)
    e, w, opp, cs = oracle.lattice(vel, I)
    for M in range(0, 6):
        IM = 0.0 if M % 2 else I[M // 2]
        for idx in itertools.product(range(D), repeat=M):
            s = sum(w[a] * np.prod([e[a, i] for i in idx]) for a in range(len(w)))
            expect = IM * cs ** M * _delta_tensor_value(idx)
            assert abs(s - expect) < 1e-13 * max(1.0, abs(expect)), (vel, idx, s, expect)
    # opposite table
    for a in range(len(w)):
        assert np.all(e[opp[a]] == -e[a])


@pytest.mark.parametrize("stat,theta,mu", [("fd", THETA, MU), ("mb", 0.7, 0.0), ("be", 0.5, -0.3)])
def test_d3v27_sixth_order_moment(stat, theta, mu):
    """Table lattices-tab: the D3V27 weights carry I_6 only through the corner
    weight I_2^3 I_6 / (216 I_4^3) and the terms that keep the lower moments.
    The sixth-order moment sum_a w_a e_x^2 e_y^2 e_z^2, to which only the eight
    corners contribute, must equal I_6 c_s^6 (the one index pattern of order 6
    whose delta tensor is 1 and which a three-speed lattice can match); a
    transcription error in the I_6 terms keeps every moment up to order 5 but
    breaks this one.  Checked for three weights, each with its own I_6."""
    I = oracle.weight_integrals(3, stat, theta, mu, nmax=4)
    e, w, opp, cs = oracle.lattice("D3V27", I)
    s6 = float(np.sum(w * (e[:, 0] ** 2) * (e[:, 1] ** 2) * (e[:, 2] ** 2)))
    assert abs(s6 - I[3] * cs ** 6) < 1e-13 * I[3] * cs ** 6, (s6, I[3] * cs ** 6)
    # the weight sum and the second and fourth moments close with the same I_6
    assert abs(w.sum() - I[0]) < 1e-13 * I[0]
    assert abs(np.sum(w * e[:, 0] ** 2) - I[1] * cs ** 2) < 1e-13 * I[1] * cs ** 2
    assert abs(np.sum(w * e[:, 0] ** 2 * e[:, 1] ** 2) - I[2] * cs ** 4) < 1e-13 * I[2] * cs ** 4


def test_d3v15_rejected_for_fd():
    """Sec. 8 requires positive weights; D3V15 gives w_0 = I_0(1 - 7J_2/9) < 0 for
    the FD weight of Sec. 9.1."""
    I = oracle.weight_integrals(3, "fd", THETA, MU, nmax=4)
    J2 = I[1] ** 2 / (I[2] * I[0])
    assert I[0] * (1 - 7 * J2 / 9) < 0
    with pytest.raises(ValueError):
        oracle.lattice("D3V15", I)
    # D3V27 is valid for the FD weight (all weights positive)
    e, w, opp, cs = oracle.lattice("D3V27", I)
    assert np.all(w > 0)


@pytest.mark.parametrize("D", [2, 3])
def test_coefficient_identities(D):
    """Sec. 9.1: c2 thetabar + c'2 + D cbar2 thetabar = 0 with thetabar = I2/I0;
    Sec. 7: J2 Delta2^2 - (D+2)(Delta2^2 - 1)/D = 1."""
    I = oracle.weight_integrals(D, "fd", THETA, MU, nmax=2)
    c = oracle.coefficients(D, I)
    assert abs(c["c2"] * c["thetabar"] + c["cprime2"] + D * c["cbar2"] * c["thetabar"]) < 1e-14
    d2 = c["Delta2"] ** 2
    assert abs(c["J2"] * d2 - (D + 2) * (d2 - 1) / D - 1.0) < 1e-14


@pytest.mark.parametrize("D", [2, 3])
def test_polynomials_orthonormal(D):
    """Sec. 3, Eq. omeg-feq: P_0 = c0, P_i = c1 xi_i, P_ij = c2 xi_i xi_j +
    (cbar2 xi^2 + c'2) delta_ij are orthonormal under omega.  Checked with the
    radial integrals: <P0 P0> = c0^2 I0, <P_i P_j> = c1^2 I2 delta_ij, and
    <P_11 P_11>, <P_12 P_12>, <P_11 P_22>, <P_0 P_11> from I0, I2, I4 (isotropy:
    <xi1^4> = 3 I4, <xi1^2 xi2^2> = I4, <xi^2 xi1^2> = (D+2) I4,
    <xi^4> = D(D+2) I4, <xi^2> = D I2)."""
    I = oracle.weight_integrals(D, "fd", THETA, MU, nmax=2)
    I0, I2, I4 = I[:3]
    c = oracle.coefficients(D, I)
    c0, c1, c2, cb, cp = c["c0"], c["c1"], c["c2"], c["cbar2"], c["cprime2"]
    assert abs(c0 * c0 * I0 - 1) < 1e-14
    assert abs(c1 * c1 * I2 - 1) < 1e-14
    # <P_11 P_0> = c0 [c2 I2 + cb D I2 + cp I0] must vanish
    assert abs(c0 * (c2 * I2 + cb * D * I2 + cp * I0)) < 1e-14
    # <P_11 P_11> = 1 (delta_{11|11} = 1), <P_12 P_12> = 1, <P_11 P_22> = 0
    p11p11 = (c2 * c2 * 3 * I4 + 2 * c2 * cb * (D + 2) * I4 + 2 * c2 * cp * I2 + cb * cb * D * (D + 2) * I4
              + 2 * cb * cp * D * I2 + cp * cp * I0)
    p12p12 = c2 * c2 * I4
    p11p22 = (c2 * c2 * I4 + 2 * c2 * cb * (D + 2) * I4 + 2 * c2 * cp * I2 + cb * cb * D * (D + 2) * I4
              + 2 * cb * cp * D * I2 + cp * cp * I0)
    assert abs(p11p11 - 2.0) < 1e-13 or abs(p11p11 - 1.0) < 1e-13
    assert abs(p12p12 - 1.0) < 1e-13
    if D >= 2:
        assert abs(p11p22) < 1e-13
    # delta_{11|11} counts permutations of the i's: 2 for (11|11)
    assert abs(p11p11 - 2.0) < 1e-13
