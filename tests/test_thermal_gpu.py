"""GPU parity of the 1D thermal model (fourth-order EDF of Sec. 4 on D1V5/D1V7,
App. A) through the C ABI against the FP64 oracle (oracle.Thermal).

Tolerances, relative L-inf on rho, j and the energy sum f xi^2: FP32 storage
1e-5; FP16/BF16 deviation storage 2e-3, or where the format cannot reach it
1.25 times its floor on the same case (the oracle with its stored deviations
rounded to the format after every step)."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import FLOOR_FACTOR, STORE_SCALE, TOL, rel_linf, round_bf16, round_f16

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WEIGHTS = {"mb": ("mb", 1.0, 0.0), "fd03": ("fd", 0.3, 1.0), "be": ("be", 0.5, -0.3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


def _fields(n, seed, thw, amp=0.02):
    rho = (1.0 + amp * (wl.uniform01(seed, n) - 0.5)).astype(np.float32)
    u = (0.02 * wl.normal(seed + 1, n)).astype(np.float32)
    th = (thw * (1.0 + amp * (wl.uniform01(seed + 2, n) - 0.5))).astype(np.float32)
    return rho, u, th


def _gpu(lattice, weight, n, tau, E, order, storage, steps, fields, seed=0):
    from paper_1710_09472_gb300.lbm import Thermal

    stat, theta, mu = WEIGHTS[weight]
    t = Thermal(lattice, n, tau, E=E, order=order, storage=storage, stat=stat, theta=theta, mu=mu)
    if storage != "f32" and seed:
        t.set_rounding(True, seed)
    dev = torch.device("cuda")
    t.init(*[torch.from_numpy(a).to(dev) for a in fields])
    t.step(steps)
    r, j, e = (torch.empty(n, device=dev) for _ in range(3))
    tot = t.moments(r, j, e)
    torch.cuda.synchronize()
    return r.cpu().numpy(), j.cpu().numpy(), e.cpu().numpy(), tot, t


def _oracle(lattice, weight, tau, E, order, steps, fields):
    stat, theta, mu = WEIGHTS[weight]
    m = oracle.Thermal(lattice, stat, theta, mu, tau=tau, E=E, order=order)
    f = m.init_state(*[a.astype(np.float64) for a in fields])
    m.step(f, steps)
    r, j, e, tot = m.moments(f)
    return r, j, e, tot, m, f


def _floor(lattice, weight, tau, E, order, steps, fields, storage, seed):
    """The oracle with its stored deviations rounded to `storage` after every
    step (stochastic, seeded; the initial state to nearest)."""
    stat, theta, mu = WEIGHTS[weight]
    m = oracle.Thermal(lattice, stat, theta, mu, tau=tau, E=E, order=order)
    rnd = {"f16": round_f16, "bf16": round_bf16}[storage]
    s = STORE_SCALE[storage]
    rng = np.random.default_rng(seed)
    f = m.init_state(*[a.astype(np.float64) for a in fields])
    n = fields[0].size
    f0 = (m.w / m.I[0])[:, None]
    f2 = f.reshape(m.Q, n)
    f2[:] = f0 + rnd(s * (f2 - f0)) / s
    for _ in range(steps):
        m.step(f, 1)
        f2[:] = f0 + rnd(s * (f2 - f0), rng) / s
    return m.moments(f)[:3]


def test_constants_match_oracle():
    """Weights, c_s, g and the 17 coefficients of the library (FP64 host
    code, its own root finder and coefficient formulas) equal the oracle's."""
    from paper_1710_09472_gb300.lbm import Thermal

    for lattice in ("D1V5b", "D1V7", "D1V7r1"):
        for weight in ("mb", "fd03", "be"):
            stat, theta, mu = WEIGHTS[weight]
            try:
                m = oracle.Thermal(lattice, stat, theta, mu, tau=0.8)
            except ValueError:
                with pytest.raises(Exception):
                    Thermal(lattice, 16, 0.8, stat=stat, theta=theta, mu=mu)
                continue
            t = Thermal(lattice, 16, 0.8, stat=stat, theta=theta, mu=mu)
            assert t.Q == m.Q
            assert abs(t.const["cs"] / m.cs - 1) < 1e-12
            assert abs(t.const["g"] / m.g - 1) < 1e-12
            np.testing.assert_allclose(t.w, m.w, rtol=1e-12, atol=0)
            lib = [t.const[k] for k in ("c0", "c1", "c2", "c3", "c4", "cp2", "cp3", "cp4", "cb2", "cb3", "cb4",
                                        "d4", "d4p", "d4b")]
            np.testing.assert_allclose(lib, m.co[:14], rtol=1e-11, atol=1e-14)
            t.close()
    # the strongly degenerate FD weight of Sec. 9.1: D1V5 root a has w_0 < 0
    with pytest.raises(Exception):
        Thermal("D1V5a", 16, 0.8)


# The FD weight at theta = 0.3 is far from Gaussian (g = 0.70): its
# third-order truncation is unstable on D1V7 (the FP64 oracle blows up within
# 400 steps from these fields), so it is run at orders 2 and 4 only, and for
# 100 steps: its random start flow decays ten times faster than the signal
# the relative error is taken against, and in FP64 already a 1e-7 change of
# the start state moves j by 2e-6 of its final size after 200 steps.
CASES = ([(lat, w, order, E, n, 200) for (lat, w) in (("D1V7", "mb"), ("D1V7", "be"), ("D1V5b", "mb"))
          for order in (4, 3, 2) for (E, n) in ((0.0, 300), (2e-4, 256))]
         + [("D1V7", "fd03", order, E, n, 100) for order in (4, 2) for (E, n) in ((0.0, 300), (2e-4, 256))])


@pytest.mark.parametrize("lattice,weight,order,E,n,steps", CASES)
def test_thermal_parity_f32(lattice, weight, order, E, n, steps):
    """FP32 storage from random rho, u, thetabar fields: rho, j and energy
    against the oracle to 1e-5, and the FP64 totals: mass and energy
    conserved (E = 0), momentum grown by rho E per step."""
    try:
        oracle.Thermal(lattice, *WEIGHTS[weight])
    except ValueError:
        pytest.skip("no such lattice for this weight")
    tau = 0.8
    m = oracle.Thermal(lattice, *WEIGHTS[weight], tau=tau)
    fields = _fields(n, 21, m.I[1] / m.I[0])
    rg, jg, eg, tg, t = _gpu(lattice, weight, n, tau, E, order, "f32", steps, fields)
    ro, jo, eo, to, m, _ = _oracle(lattice, weight, tau, E, order, steps, fields)
    er, ej, ee = rel_linf(rg, ro), rel_linf(jg, jo), rel_linf(eg, eo)
    print(f"thermal {lattice} {weight} order {order} E {E} {steps} steps: rho {er:.2e} j {ej:.2e} energy {ee:.2e}")
    assert er <= 1e-5 and ej <= 1e-5 and ee <= 1e-5, (er, ej, ee)
    assert abs(tg[0] / to[0] - 1) < 1e-6 and abs(tg[2] / to[2] - 1) < 1e-6
    assert abs(tg[1] - to[1]) < 1e-5 * max(abs(to[1]), to[0] * 0.02)
    t.close()


@pytest.mark.parametrize("lattice,weight", [("D1V7", "mb"), ("D1V5b", "mb"), ("D1V7", "be")])
def test_thermal_parity_long_row(lattice, weight):
    """A row of 2309 cells (FP32, order 4, with force): the blocks away from
    both ends pull at fixed offsets without the periodic wrap, the two end
    blocks with it.  After 150 steps every population is within 1e-6 of the
    largest population, and rho, j and energy within 1e-5."""
    n, tau, E, order, steps = 2309, 0.8, 1e-4, 4, 150
    m = oracle.Thermal(lattice, *WEIGHTS[weight], tau=tau, E=E)
    fields = _fields(n, 51, m.I[1] / m.I[0])
    rg, jg, eg, _, t = _gpu(lattice, weight, n, tau, E, order, "f32", steps, fields)
    f = torch.empty(t.Q * n, device="cuda")
    t.populations(f)
    fg = f.cpu().numpy().astype(np.float64).reshape(t.Q, n)
    t.close()
    ro, jo, eo, _, _, fo = _oracle(lattice, weight, tau, E, order, steps, fields)
    fo = fo.reshape(m.Q, n)
    assert np.max(np.abs(fg - fo)) <= 1e-6 * np.max(np.abs(fo))
    er, ej, ee = rel_linf(rg, ro), rel_linf(jg, jo), rel_linf(eg, eo)
    assert er <= 1e-5 and ej <= 1e-5 and ee <= 1e-5, (er, ej, ee)


def test_populations_elementwise():
    """Every population after 7 steps (FP32 storage, D1V7, order 4)."""
    m = oracle.Thermal("D1V7", *WEIGHTS["fd03"], tau=0.7, E=1e-4)
    n = 130
    fields = _fields(n, 31, m.I[1] / m.I[0])
    _, _, _, _, t = _gpu("D1V7", "fd03", n, 0.7, 1e-4, 4, "f32", 7, fields)
    f = torch.empty(t.Q * n, device="cuda")
    t.populations(f)
    fg = f.cpu().numpy().astype(np.float64).reshape(t.Q, n)
    _, _, _, _, _, fo = _oracle("D1V7", "fd03", 0.7, 1e-4, 4, 7, fields)
    fo = fo.reshape(m.Q, n)
    assert np.max(np.abs(fg - fo)) <= 2e-7 * np.max(np.abs(fo))
    t.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_thermal_parity_16bit(storage):
    """FP16/BF16 deviation storage, D1V7, MB weight, 400 steps."""
    lattice, weight, tau, E, order, steps, n = "D1V7", "mb", 0.8, 2e-4, 4, 400, 512
    m = oracle.Thermal(lattice, *WEIGHTS[weight], tau=tau)
    fields = _fields(n, 41, m.I[1] / m.I[0])
    rg, jg, eg, tg, t = _gpu(lattice, weight, n, tau, E, order, storage, steps, fields)
    t.close()
    ro, jo, eo, to, _, _ = _oracle(lattice, weight, tau, E, order, steps, fields)
    errs = (rel_linf(rg, ro), rel_linf(jg, jo), rel_linf(eg, eo))
    floors = [0.0, 0.0, 0.0]
    if max(errs) > TOL[storage]:
        for sd in (1, 2, 3):
            fr = _floor(lattice, weight, tau, E, order, steps, fields, storage, sd)
            for k, (a, b) in enumerate(zip(fr, (ro, jo, eo))):
                floors[k] = max(floors[k], rel_linf(a, b))
    bounds = [max(TOL[storage], FLOOR_FACTOR * fl) for fl in floors]
    print(f"thermal {storage}: errors {errs}, floors {floors}, bounds {bounds}")
    assert all(e <= b for e, b in zip(errs, bounds)), (errs, floors)


def test_thermal_sound_speed_on_gpu():
    """The adiabatic sound speed of the model, c = c_s sqrt(3 thetabar) in
    lattice units (the linearised mass, momentum and energy equations in 1D),
    measured from a standing wave run through the C ABI (FP32, D1V7, FD
    weight theta = 0.3): within 1e-3 of the formula, and far from the
    isothermal c_s sqrt(thetabar)."""
    from paper_1710_09472_gb300.lbm import Thermal

    stat, theta, mu = WEIGHTS["fd03"]
    n, steps = 256, 700
    t = Thermal("D1V7", n, 0.8, stat=stat, theta=theta, mu=mu)
    thw = t.const["thetabar_w"]
    x = np.arange(n)
    k = 2 * np.pi / n
    dev = torch.device("cuda")
    rho = torch.from_numpy((1.0 + 1e-4 * np.cos(k * x)).astype(np.float32)).to(dev)
    t.init(rho, None, None)
    j = torch.empty(n, device=dev)
    probe = []
    for _ in range(steps):
        t.step(1)
        t.moments(None, j, None, totals=False)
        probe.append(float(j[n // 4]))
    probe = np.array(probe)
    s = np.sign(probe)
    cross = np.flatnonzero(s[1:] != s[:-1])
    tc = [c + probe[c] / (probe[c] - probe[c + 1]) for c in cross]
    c = (2 * np.pi / (2 * float(np.mean(np.diff(tc))))) / k
    want = t.const["cs"] * math.sqrt(3 * thw)
    print(f"sound speed {c:.6f} vs {want:.6f} (isothermal {t.const['cs'] * math.sqrt(thw):.6f})")
    assert abs(c / want - 1) < 1e-3
    t.close()


def test_thermal_errors():
    from paper_1710_09472_gb300._lib import LBMError
    from paper_1710_09472_gb300.lbm import Thermal

    with pytest.raises(LBMError):
        Thermal("D1V7", 16, 0.5)  # tau must exceed 1/2
    with pytest.raises(LBMError):
        Thermal("D1V7", 16, 0.8, order=5)
    t = Thermal("D1V7", 16, 0.8, stat="mb", theta=1.0, mu=0.0)
    with pytest.raises(LBMError):
        t.step(1)  # before init: LBM_ERR_STATE
    with pytest.raises(LBMError):
        t.set_rounding(True)  # FP32 storage
    t.init()
    t.step(3)
    tot = t.moments()
    assert abs(tot[0] - 16.0) < 1e-5
    t.close()
