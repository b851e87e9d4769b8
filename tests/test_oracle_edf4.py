"""Pins of the oracle's fourth-order equilibrium (Sec. 3 coefficients up to
K = 4, Sec. 4 projections and Eq. feq-4order-01), of the D1V5/D1V7 lattices
(Table lattices-tab, App. A) and of the 1D thermal model built on them.  CPU
only.

The pins do not retype the oracle's formulas: the coefficients are checked by
the orthonormality that defines them (Eq. omeg-feq), the projections by the
integral that defines them, the lattices by their quadrature equations, the
EDF by the exact moments a fourth-order expansion must keep, and the thermal
model by conservation and by its sound speed."""
import itertools
import math

import numpy as np
import pytest

import oracle

THETA = 1.0 / 270.0

# (D, weight, theta, mu): FD and BE are far from the Hermite weight, MB at
# theta != 1 is a scaled Hermite weight
WEIGHTS = [(1, "fd", 0.3, 1.0), (1, "fd", THETA, 1.0), (2, "fd", 0.25, 1.0), (3, "fd", 0.3, 1.0),
           (3, "be", 0.5, -0.3), (2, "mb", 0.7, 0.0)]


def _dfact(n):
    return 1 if n <= 0 else n * _dfact(n - 2)


def _sym_polys(D, co, xs):
    """The Sec. 3 tensor polynomials built from the coefficients `co` (as
    returned by oracle.coefficients4) on sympy symbols xs."""
    c = co[0:5]
    cp = {2: co[5], 3: co[6], 4: co[7]}
    cb = {2: co[8], 3: co[9], 4: co[10]}
    d4, d4p, d4b = co[11], co[12], co[13]
    x2 = sum(v * v for v in xs)
    dl = lambda i, j: 1 if i == j else 0  # noqa: E731
    f2, f3, f4 = cb[2] * x2 + cp[2], cb[3] * x2 + cp[3], cb[4] * x2 + cp[4]
    g4 = d4b * x2 ** 2 + d4p * x2 + d4
    P = {(): c[0]}
    for i in range(D):
        P[(i,)] = c[1] * xs[i]
    for i, j in itertools.product(range(D), repeat=2):
        P[(i, j)] = c[2] * xs[i] * xs[j] + f2 * dl(i, j)
    for i, j, k in itertools.product(range(D), repeat=3):
        P[(i, j, k)] = c[3] * xs[i] * xs[j] * xs[k] + f3 * (xs[i] * dl(j, k) + xs[j] * dl(i, k) + xs[k] * dl(i, j))
    for i, j, k, l in itertools.product(range(D), repeat=4):
        six = (xs[i] * xs[j] * dl(k, l) + xs[i] * xs[k] * dl(j, l) + xs[i] * xs[l] * dl(j, k)
               + xs[j] * xs[k] * dl(i, l) + xs[j] * xs[l] * dl(i, k) + xs[k] * xs[l] * dl(i, j))
        P[(i, j, k, l)] = (c[4] * xs[i] * xs[j] * xs[k] * xs[l] + f4 * six
                           + g4 * (dl(i, j) * dl(k, l) + dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k)))
    return P


def _moment_integral(sp, expr, xs, mom):
    """int d^D xi w(xi) expr(xi) for a polynomial expr, from the isotropic
    moments int w xi_1^a1 .. xi_D^aD = mom[(a1+..+aD)/2] prod (a_k - 1)!!
    (Sec. 3, Eq. i2n-cont: I_N delta_{i1..iN}; the delta tensor of an index
    multiset with counts a_k is the number of its pairings)."""
    poly = sp.Poly(sp.expand(expr), *xs)
    tot = 0.0
    for mon, coef in poly.terms():
        if any(m % 2 for m in mon):
            continue
        tot += float(coef) * mom[sum(mon) // 2] * np.prod([_dfact(m - 1) for m in mon])
    return tot


def _perm_delta(a, b):
    """delta_{i1..iN | j1..jN}: the number of permutations mapping a onto b."""
    if len(a) != len(b):
        return 0
    return sum(1 for p in itertools.permutations(range(len(b))) if all(a[t] == b[p[t]] for t in range(len(a))))


@pytest.mark.parametrize("D,stat,theta,mu", WEIGHTS)
def test_polynomials_orthonormal(D, stat, theta, mu):
    """Eq. omeg-feq: int w P_{i..} P_{j..} = delta_NM delta_{i..|j..} for every
    pair of index tuples up to order 4, with the polynomials built from the
    oracle's 17 coefficients; and the oracle's own P_N evaluate to the same
    tensors at random points."""
    sp = pytest.importorskip("sympy")
    I = oracle.weight_integrals(D, stat, theta, mu, nmax=4)
    co = oracle.coefficients4(D, I)
    xs = sp.symbols("x0:%d" % D)
    P = _sym_polys(D, co, xs)
    keys = [k for k in P if list(k) == sorted(k)]
    worst = 0.0
    for a in keys:
        for b in keys:
            if len(b) < len(a):
                continue
            val = _moment_integral(sp, P[a] * P[b], xs, I)
            want = _perm_delta(a, b) if len(a) == len(b) else 0
            worst = max(worst, abs(val - want))
    assert worst < 1e-11, worst
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.normal(0, 0.7, D)
        got = oracle.polynomials(D, co, x)
        for k, expr in P.items():
            v = float(expr.subs(dict(zip(xs, x)))) if not isinstance(expr, float) else expr
            assert abs(got[len(k)][k] - v) < 1e-12 * max(1.0, abs(v)), (k, got[len(k)][k], v)


def test_hermite_limit_coefficients():
    """Sec. 3: with I_2N = 1 (the Hermite weight), c_K = 1, cbar_K = 0,
    c'_K = -1, d_4 = 1, dbar_4 = 0 and d'_4 = 0, in every dimension."""
    for D in (1, 2, 3):
        co = dict(zip(oracle.COEF4_KEYS, oracle.coefficients4(D, np.ones(5))))
        for K in range(5):
            assert abs(co[f"c{K}"] - 1) < 1e-15
        for K in (2, 3, 4):
            assert abs(co[f"cp{K}"] + 1) < 1e-15 and abs(co[f"cb{K}"]) < 1e-15
        assert abs(co["d4"] - 1) < 1e-15 and abs(co["d4p"]) < 1e-15 and abs(co["d4b"]) < 1e-15


@pytest.mark.parametrize("D,stat,theta,mu", [w for w in WEIGHTS if w[1] != "mb"])
def test_projections_match_definition(D, stat, theta, mu):
    """Sec. 4: A_{i1..iN}(u) = int d^D eta f^eq(eta) P_{i1..iN}(eta + u) for an
    isotropic f^eq with int f = rho, int f eta_i eta_j = rho thetabar delta_ij
    and int f eta_i eta_j eta_k eta_l = rho thetabar^2 g delta_ijkl
    (Eq. int-2nd-coeff-eq).  The oracle's A_0..A_4 (the printed closed forms)
    against that integral at random rho, u, thetabar, g."""
    sp = pytest.importorskip("sympy")
    I = oracle.weight_integrals(D, stat, theta, mu, nmax=4)
    co = oracle.coefficients4(D, I)
    rng = np.random.default_rng(5)
    rho, u, th, g = 1.3, rng.normal(0, 0.2, D), 0.37, 1.21
    eta = sp.symbols("e0:%d" % D)
    P = _sym_polys(D, co, [eta[i] + u[i] for i in range(D)])
    A = oracle.projections(D, co, rho, u, th, g)
    mom = {0: rho, 1: rho * th, 2: rho * th * th * g}
    for k, expr in P.items():
        want = _moment_integral(sp, expr, eta, mom)
        assert abs(A[len(k)][k] - want) < 1e-12 * max(1.0, abs(want)), (k, A[len(k)][k], want)


@pytest.mark.parametrize("stat,theta,mu", [("fd", THETA, 1.0), ("fd", 0.1, 1.0), ("mb", 1.0, 0.0),
                                           ("mb", 0.5, 0.0), ("be", 0.5, -0.3)])
def test_lattice1d_quadrature(stat, theta, mu):
    """Sec. 8, Eq. quadrature-eq-2 in 1D: sum_a w_a e_a^{2k} = (2k - 1)!! I_2k c_s^{2k}
    up to the lattice's order (D1V5: M = 7, k <= 3; D1V7: M = 9, k <= 4), odd
    moments zero, weights positive.  The D1V7 root 0 equals the closed form
    printed in App. A."""
    I = oracle.weight_integrals(1, stat, theta, mu, nmax=4)
    for kind, kmax in (("D1V5a", 3), ("D1V5b", 3), ("D1V7", 4), ("D1V7r1", 4)):
        try:
            e, w, cs = oracle.lattice1d(kind, I)
        except ValueError:
            continue  # a root with a non-positive weight is rejected (Sec. 8)
        assert np.all(w > 0) and cs > 0
        for k in range(kmax + 1):
            s = float(np.sum(w * e.astype(float) ** (2 * k)))
            want = _dfact(2 * k - 1) * I[k] * cs ** (2 * k)
            assert abs(s - want) < 1e-12 * want, (kind, k, s, want)
            assert abs(float(np.sum(w * e.astype(float) ** (2 * k + 1)))) < 1e-14
    I0, I2, I4, I6, I8 = I
    A = -4900 * I6 ** 2 + 5145 * I4 * I8
    B = 686000 * I6 ** 3 - 1080450 * I4 * I6 * I8 + 396900 * I2 * I8 ** 2
    R = (B + np.sqrt(complex(4 * A ** 3 + B ** 2))) ** (1 / 3)
    cs_printed = np.sqrt(2 / 3 * I6 / I8 - 49 * 2 ** (1 / 3) * I4 / R + 140 * 2 ** (1 / 3) * I6 ** 2 / (3 * I8 * R)
                         + R / (105 * 2 ** (1 / 3) * I8))
    assert abs(cs_printed.imag) < 1e-9
    assert abs(oracle.lattice1d("D1V7", I)[2] / cs_printed.real - 1) < 1e-9


def test_d1v5a_rejected_for_fd():
    """Table lattices-tab, D1V5 with the + root: w_0 < 0 for the FD weight of
    Sec. 9.1, so Sec. 8 rejects it; the - root (D1V5b) is admissible."""
    I = oracle.weight_integrals(1, "fd", THETA, 1.0, nmax=4)
    with pytest.raises(ValueError):
        oracle.lattice1d("D1V5a", I)
    assert np.all(oracle.lattice1d("D1V5b", I)[1] > 0)


@pytest.mark.parametrize("kind,kmax", [("D1V7", 4), ("D1V7r1", 4), ("D1V5b", 3)])
@pytest.mark.parametrize("stat,theta,mu", [("fd", THETA, 1.0), ("mb", 1.0, 0.0), ("be", 0.5, -0.3)])
def test_edf4_discrete_moments(kind, kmax, stat, theta, mu):
    """A fourth-order expansion keeps the moments of the shifted EDF up to
    order 4; on a lattice of order M the discrete sums are exact up to order
    M - 4 - ... so on D1V7 (M = 9) sum_a f^eq_a xi_a^k for k <= 4 equals
    rho, rho u, rho (thb + u^2), rho (u^3 + 3 thb u), rho (u^4 + 6 thb u^2 +
    3 g thb^2) (1D: delta_1111 = 3); on D1V5 (M = 7) for k <= 3."""
    try:
        m = oracle.Thermal(kind, stat, theta, mu, tau=0.8)
    except ValueError:
        pytest.skip(f"{kind} has no admissible root for this weight")
    rng = np.random.default_rng(7)
    for _ in range(4):
        rho, u, th = 1.0 + 0.1 * rng.random(), 0.15 * rng.normal(), m.I[1] / m.I[0] * (1 + 0.2 * rng.normal())
        f = m.equilibrium(rho, u, th)
        want = [rho, rho * u, rho * (th + u * u), rho * (u ** 3 + 3 * th * u),
                rho * (u ** 4 + 6 * th * u * u + 3 * m.g * th * th)]
        for k in range(kmax + 1):
            got = float(np.sum(f * m.xi ** k))
            assert abs(got - want[k]) < 1e-12 * max(1.0, abs(want[k])), (kind, k, got, want[k])


def test_edf_second_order_is_the_direct_form():
    """Sec. 4 truncated at N = 2 with thetabar = I_2/I_0 equals the direct N = 2
    form of Sec. 5.1 (Eq. feq-reduce-general-method-without-pol-eq):
    rho w/I_0 {1 + (I_0/I_2) xi.u + (I_0/2I_4)(xi.u)^2
               + u^2/2 [(I_0/I_4)((Delta_2^2 - 1)/D) xi^2 - (I_2/I_4) Delta_2^2]}."""
    for D, stat, theta, mu in [(1, "fd", THETA, 1.0), (2, "fd", 0.25, 1.0), (3, "be", 0.5, -0.3)]:
        I = oracle.weight_integrals(D, stat, theta, mu, nmax=4)
        co = oracle.coefficients4(D, I)
        I0, I2, I4 = I[:3]
        J2 = I2 * I2 / (I4 * I0)
        d2 = 2.0 / ((D + 2) - J2 * D)  # Delta_2^2
        rng = np.random.default_rng(11)
        for _ in range(5):
            xi, u, rho = rng.normal(0, 1.0, D), rng.normal(0, 0.1, D), 1.1
            got = oracle.edf(D, 2, co, 1.0, xi, rho, u, I2 / I0, 1.0)
            xu, u2, x2 = float(xi @ u), float(u @ u), float(xi @ xi)
            want = rho / I0 * (1 + I0 / I2 * xu + I0 / (2 * I4) * xu * xu
                               + 0.5 * u2 * (I0 / I4 * (d2 - 1) / D * x2 - I2 / I4 * d2))
            assert abs(got - want) < 1e-13 * max(1.0, abs(want)), (D, got, want)


@pytest.mark.parametrize("kind", ["D1V7", "D1V7r1", "D1V5b"])
def test_thermal_collision_invariants(kind):
    """The collision keeps mass and energy and changes the momentum by rho E
    (Sec. 7 velocity shift, u* = u + tau E): sum f* = sum f,
    sum f* xi = sum f xi + rho E, sum f* xi^2 = sum f xi^2 + (rho/tau)(u*^2 - u^2)."""
    m = oracle.Thermal(kind, "fd", THETA, 1.0, tau=0.8, E=3e-3)
    rng = np.random.default_rng(13)
    for _ in range(5):
        f = m.equilibrium(1.0 + 0.05 * rng.random(), 0.05 * rng.normal(), m.I[1] / m.I[0] * 1.05)
        f = f * (1 + 0.01 * rng.normal(size=m.Q))
        fo = m.collide_cell(f)
        rho, j, e2 = f.sum(), f @ m.xi, f @ m.xi ** 2
        u = j / rho
        us = u + m.tau * m.E
        assert abs(fo.sum() - rho) < 1e-14 * rho
        assert abs(fo @ m.xi - (j + rho * m.E)) < 1e-14 * max(1.0, abs(j))
        assert abs(fo @ m.xi ** 2 - (e2 + rho / m.tau * (us * us - u * u))) < 1e-13 * e2


def _sound_speed(m, n=256, steps=700, amp=1e-4):
    """Speed of a standing sound wave: rho = 1 + amp cos(k x), u = 0,
    thetabar uniform; returns the measured speed (lattice units per step)
    from the zero crossings of j at x = n/4 (where it is largest)."""
    x = np.arange(n)
    k = 2 * np.pi / n
    th0 = m.I[1] / m.I[0]
    f = m.init_state(1.0 + amp * np.cos(k * x), 0.0, th0)
    probe = []
    for _ in range(steps):
        m.step(f, 1)
        probe.append(m.moments(f)[1][n // 4])
    probe = np.array(probe)
    s = np.sign(probe)
    cross = np.flatnonzero(s[1:] != s[:-1])
    t = [c + probe[c] / (probe[c] - probe[c + 1]) for c in cross]  # linear interpolation
    half_periods = np.diff(t)
    period = 2 * float(np.mean(half_periods))
    return (2 * np.pi / period) / k, th0


@pytest.mark.parametrize("stat,theta,mu", [("mb", 1.0, 0.0), ("fd", 0.3, 1.0), ("be", 0.5, -0.3)])
def test_thermal_sound_speed(stat, theta, mu):
    """Linearising the moment equations of the thermal model (mass, momentum
    and energy, with the pressure rho thetabar of Sec. 4) gives the adiabatic
    sound speed c^2 = 3 thetabar in 1D (xi units); the isothermal model of
    Sec. 9.1 has c^2 = thetabar.  The measured speed of a standing wave on
    D1V7 (lattice units c_s sqrt(3 thetabar)) agrees to 1e-3 for the Hermite,
    a mildly degenerate FD and a BE weight.  (With the strongly degenerate FD
    weight of Sec. 9.1, theta = 1/270, the thermal sound speed is c_s = 2.3 or
    3.3 cells per step on the two admissible D1V7 roots, against the
    lattice's largest speed 3, and the model does not run stably.)"""
    m = oracle.Thermal("D1V7", stat, theta, mu, tau=0.8)
    c, th0 = _sound_speed(m)
    want = m.cs * math.sqrt(3 * th0)
    assert abs(c / want - 1) < 1e-3, (c, want, m.cs * math.sqrt(th0))
