"""The porous and differentiable workloads at their stated sizes, on the GPU,
against the FP64 oracle (sampled one-step checks, light-cone sub-boxes) and
against what the physics fixes (Ohm's law, Hall current, conservation,
central finite differences).

- Porous 256^3 (spheres r = 6, porosity 0.7, seed 1, D3V19, tau = 0.8), the
  Ohm experiment of Sec. 9.4 run as a sweep: E_x in {1, 2, 4, 8} 1e-6 and
  B_z in {0, 1e-3}, 20000 steps, FP32 and FP16-deviation storage.
- Differentiable porous 1024^2 (disks r = 8, porosity 0.6, per-cell E_x ~
  N(1e-6, 1e-7), tau = 0.7), 4000 steps, loss = total x-current over the last
  500 steps, checkpoints every 100 steps: the adjoint against central
  differences of the FP32 forward.
- Porous 512^3 (spheres r = 10, porosity 0.65, seed 5, E_x = 2e-6, B_z = 5e-4),
  the first 200 steps: sampled one-step checks at steps 1 and 200 and the
  oracle on a light-cone sub-box after 100 steps.
"""
import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import (THETA, deviations_on_device, light_cone_oracle, one_step_sampled, rel_linf)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


def _sim(vel, shape, solid_dev, tau, storage, E=(0, 0, 0), B=(0, 0, 0), force="term"):
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM(vel, tuple(reversed(shape)), tau, E=E, B=B, storage=storage, force=force)
    sim.set_geometry(solid_dev)
    sim.init_equilibrium()
    return sim


def _fields(sim):
    rho = torch.empty(sim.N, dtype=torch.float32, device="cuda")
    j = torch.empty(sim.D * sim.N, dtype=torch.float32, device="cuda")
    tot = sim.moments(rho, j)
    return rho, j, tot


def _rel_dev(a, b):
    return float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))


# ---------------------------------------------------------------------------
# Porous 256^3: Ohm's law and the Hall current (Sec. 9.4), FP32 vs FP16.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def porous256():
    w = wl.porous_3d(256, steps=20000)
    w["solid_dev"] = torch.from_numpy(w["solid"].reshape(-1)).cuda()
    return w


E_SWEEP = (1e-6, 2e-6, 4e-6, 8e-6)


@pytest.mark.parametrize("Bz", [0.0, 1e-3])
def test_porous256_ohm_hall_sweep(porous256, Bz):
    """20000 steps per run.  <j_x>/E is the same for every E to 1e-4 (Ohm's
    law; the nonlinearity is O(u^2)), and so is <j_y>/E to 1e-4 of <j_x>/E
    (with B_z = 1e-3 the Hall current, linear to 1e-3 of itself; with B_z = 0
    the transverse current of the random packing).

    FP16-deviation storage against FP32 storage (itself within 1e-5 of the
    oracle on the smaller configs) at the end of every run, relative L-inf on
    rho and j: 2e-3, or 1.25 times the FP16 rounding floor where that is
    larger.  The oracle cannot run this box for 20000 steps, so the floor is
    estimated from the FP16 runs themselves: three runs that differ only in
    the rounding seed differ by their rounding noise alone, and the L-inf of
    the difference of two of them is sqrt(2) times the L-inf of one run's
    noise.  The error against FP32 is the median over the three runs, the
    floor the largest over the three pairs.  After the last FP32 run the oracle
    collides and streams its state at 3000 sampled fluid cells."""
    w = porous256
    shape, steps = w["shape"], w["steps"]
    n_fluid = int((w["solid"] == 0).sum())
    ratios, report = [], []
    last = None
    for Ex in E_SWEEP:
        res = {}
        for storage, seed in (("f32", 0), ("f16", 0), ("f16", 1), ("f16", 2)):
            sim = _sim("D3V19", shape, w["solid_dev"], w["tau"], storage, E=(Ex, 0, 0), B=(0, 0, Bz))
            if seed:
                sim.set_rounding_seed(seed)
            sim.step(steps)
            rho, j, (tr, tj) = _fields(sim)
            res[(storage, seed)] = (rho, j, tr, np.asarray(tj))
            if storage == "f32" and Ex == E_SWEEP[-1]:
                last = sim
            else:
                sim.close()
        r32, j32, tr32, tj32 = res[("f32", 0)]
        runs = [res[("f16", k)] for k in range(3)]
        er = float(np.median([_rel_dev(r[0], r32) for r in runs]))
        ej = float(np.median([_rel_dev(r[1], j32) for r in runs]))
        pairs = ((0, 1), (0, 2), (1, 2))
        fr = max(_rel_dev(runs[a][0], runs[b][0]) for a, b in pairs) / np.sqrt(2.0)
        fj = max(_rel_dev(runs[a][1], runs[b][1]) for a, b in pairs) / np.sqrt(2.0)
        br, bj = max(2e-3, 1.25 * fr), max(2e-3, 1.25 * fj)
        ratios.append((tj32[0] / n_fluid / Ex, tj32[1] / n_fluid / Ex))
        report.append((Ex, er, ej, fr, fj, br, bj))
        print(f"Bz={Bz} Ex={Ex:.0e}: <j_x>/E {ratios[-1][0]:.9e} <j_y>/E {ratios[-1][1]:.6e} "
              f"fp16 vs fp32 (median of 3 seeds) rho {er:.2e} j {ej:.2e} (rounding floor {fr:.2e} {fj:.2e}; "
              f"bound {br:.2e} {bj:.2e})")
        del res, runs
    for Ex, er, ej, fr, fj, br, bj in report:
        assert er <= br and ej <= bj, (Ex, er, ej, fr, fj)
    rx = np.array([r[0] for r in ratios])
    ry = np.array([r[1] for r in ratios])
    assert np.max(np.abs(rx / rx[0] - 1)) <= 1e-4, rx
    # the transverse current is linear in E to the same 1e-4 of the current's
    # size as <j_x> (its O(u^2) part is of the same absolute size)
    assert np.max(np.abs(ry - ry[0])) <= 1e-4 * abs(rx[0]), ry
    if Bz != 0.0:
        # the Hall current: the Lorentz force u x B pushes a current along x
        # towards -y for B_z > 0, so <j_y> is opposite to <j_x>, and it is
        # linear in E to 1e-3 of itself
        assert ry[0] * rx[0] < 0 and abs(ry[0]) > 1e-4 * abs(rx[0]), ry
        assert np.max(np.abs(ry / ry[0] - 1)) <= 1e-3, ry

    # sampled one-step check of the long run's state (E_x = 8e-6)
    sim = last
    h_t = deviations_on_device(sim)
    sim.step(1)
    h_t1 = deviations_on_device(sim)
    m = oracle.Model("D3V19", "fd", THETA, 1.0, tau=w["tau"], E=(E_SWEEP[-1], 0, 0), B=(0, 0, Bz), force="term")
    solid = w["solid"].reshape(-1)
    cells = np.random.default_rng(11).choice(np.flatnonzero(solid == 0), 3000, replace=False)
    err, scale = one_step_sampled(m, sim.dims, solid, h_t, h_t1, cells)
    print(f"one-step after {steps} steps: max err {err:.3e} of {scale:.3e}")
    assert err <= 1e-5 * scale, (err, scale)
    sim.close()


# ---------------------------------------------------------------------------
# Differentiable porous 1024^2: adjoint vs central differences.
# ---------------------------------------------------------------------------
def test_differentiable_1024_adjoint_vs_finite_differences():
    """Per-cell dL/dE_x at 32 seeded fluid cells, dL/dB_z and dL/dtau from one
    lbm_adjoint call (checkpoints every 100 steps) against central differences
    of the FP32 GPU forward: relative 1e-3.

    The per-cell step is 1e-4 (a hundred times the mean field).  A smaller
    step is lost in the FP32 forward's rounding: the two runs round
    differently in every cell the perturbation reaches, and over 4000 steps
    on 10^6 cells that noise is a few 1e-6 in L, 0.1% of the change that a
    1e-5 step makes.  A central difference cancels the even orders, and L is
    linear in E up to O(u^2), so the larger step costs no accuracy.

    For B_z and tau the central differences are Richardson-extrapolated from
    steps h and h/2, which removes their O(h^2) error: x-current is even in
    B_z up to the small part that the random packing makes odd, so the cubic
    term (relative size of the squared Hall angle, 5e-3 at B_z = 1e-3) is
    not small against the first-order one."""
    from paper_1710_09472_gb300.lbm import LBM

    w = wl.porous_2d_differentiable()
    shape, T, K = w["shape"], w["steps"], w["checkpoint_every"]
    tb = T - w["loss_window"]
    n = shape[0]
    solid_dev = torch.from_numpy(w["solid"].reshape(-1)).cuda()
    Ef = torch.from_numpy(w["Efield"].reshape(-1)).cuda()
    tau = w["tau"]

    sim = LBM("D2V9", (n, n), tau, storage="f32", force="term")
    sim.set_geometry(solid_dev)

    def loss(E_dev, tau_=tau, Bz=0.0):
        sim.set_params(tau_, B=(0.0, 0.0, Bz))
        sim.set_E_field(E_dev)
        sim.init_equilibrium()
        return float(sim.window_totals(tb, T)[1])

    sim.set_E_field(Ef)
    sim.init_equilibrium()
    wj = torch.zeros(2 * sim.N, dtype=torch.float32, device="cuda")
    wj[: sim.N] = 1.0
    dE = torch.empty(2 * sim.N, dtype=torch.float64, device="cuda")
    res = sim.adjoint(tb, T, None, wj, K, dL_dE=dE)
    st = sim.adjoint_stats()
    assert st["reverse_steps"] == T
    gE = dE.view(2, -1)[0].cpu().numpy()
    L0 = loss(Ef)
    assert abs(res["loss"] / L0 - 1) < 1e-6, (res["loss"], L0)

    cells = np.random.default_rng(4).choice(np.flatnonzero(w["solid"].reshape(-1) == 0), 32, replace=False)
    d = 1e-4
    rel = []
    for c in cells:
        Ep = Ef.clone()
        Ep[int(c)] += d
        Lp = loss(Ep)
        Ep[int(c)] -= 2 * d
        Lm = loss(Ep)
        fd = (Lp - Lm) / (2 * d)
        rel.append((int(c), gE[c], fd, abs(gE[c] / fd - 1)))
    worst = max(r[3] for r in rel)
    def richardson(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_tau = richardson(lambda dt: loss(Ef, tau + dt), 5e-3 * tau)
    fd_B = richardson(lambda b: loss(Ef, tau, b), 1e-3)
    print(f"1024^2: worst per-cell rel {worst:.2e}; dL/dtau {res['dL_dtau']:.6e} vs {fd_tau:.6e}; "
          f"dL/dB_z {res['dL_dB'][2]:.6e} vs {fd_B:.6e}; loss {L0:.6e}")
    assert worst < 1e-3, [r for r in rel if r[3] >= 1e-3]
    assert abs(res["dL_dtau"] / fd_tau - 1) < 1e-3, (res["dL_dtau"], fd_tau)
    assert abs(res["dL_dB"][2] - fd_B) < 1e-3 * max(abs(fd_B), 1e-6 * abs(L0)), (res["dL_dB"][2], fd_B)
    sim.close()


# ---------------------------------------------------------------------------
# Porous 512^3: the first 200 steps against the oracle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_porous512_first_200_steps(storage):
    """The 512^3 workload in the launch configuration of its adjoint run.

    - steps 1 and 200: the oracle collides and streams the GPU state at 2000
      sampled fluid cells (FP32: 1e-5 of the largest deviation; FP16: one
      storage ulp, 2^-9 relative, as stochastic rounding picks either
      neighbour);
    - step 100: the oracle's rho and j on a 12^3 block, run on a periodic
      sub-box with a 101-cell margin (the light cone of the block), against
      the GPU's (relative L-inf: 1e-5 FP32, 2e-3 FP16);
    - sum rho over the fluid cells is conserved over the 200 steps."""
    w = wl.porous_3d_512()
    shape = w["shape"]
    solid = w["solid"]
    solid_flat = solid.reshape(-1)
    sim = _sim("D3V19", shape, torch.from_numpy(solid_flat).cuda(), w["tau"], storage, E=w["E"], B=w["B"])
    m = oracle.Model("D3V19", "fd", THETA, 1.0, tau=w["tau"], E=w["E"], B=w["B"], force="term")
    fluid = np.flatnonzero(solid_flat == 0)
    rng = np.random.default_rng(5)
    tol = 1e-5 if storage == "f32" else 2.0 ** -9
    m0, _ = sim.moments()

    h0 = deviations_on_device(sim)
    sim.step(1)
    h1 = deviations_on_device(sim)
    err, scale = one_step_sampled(m, sim.dims, solid_flat, h0, h1, rng.choice(fluid, 2000, replace=False))
    del h0, h1
    print(f"512^3 {storage} step 1: {err:.3e} of {scale:.3e}")
    assert err <= tol * scale, (err, scale)

    sim.step(99)
    rho = torch.empty(sim.N, dtype=torch.float32, device="cuda")
    j = torch.empty(3 * sim.N, dtype=torch.float32, device="cuda")
    sim.moments(rho, j)
    corner, block = (250, 130, 500), 12
    zz, yy, xx = (np.arange(corner[d], corner[d] + block) % shape[d] for d in range(3))
    sel = torch.from_numpy(((zz[:, None, None] * shape[1] + yy[None, :, None]) * shape[2]
                            + xx[None, None, :]).reshape(-1)).cuda()
    rg = rho[sel].cpu().numpy().reshape((block,) * 3)
    jg = j.view(3, -1)[:, sel].cpu().numpy().reshape((3,) + (block,) * 3)
    del rho, j
    ro, jo, sub = light_cone_oracle(m, solid, corner, block, 100)
    assert np.array_equal(sub, solid[np.ix_(zz, yy, xx)])
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"512^3 {storage} light cone after 100 steps: rho {er:.3e} j {ej:.3e}")
    bound = 1e-5 if storage == "f32" else 2e-3
    assert er <= bound and ej <= bound, (er, ej)

    sim.step(99)
    h199 = deviations_on_device(sim)
    sim.step(1)
    h200 = deviations_on_device(sim)
    err, scale = one_step_sampled(m, sim.dims, solid_flat, h199, h200, rng.choice(fluid, 2000, replace=False))
    del h199, h200
    print(f"512^3 {storage} step 200: {err:.3e} of {scale:.3e}")
    assert err <= tol * scale, (err, scale)
    m1, _ = sim.moments()
    assert abs(m1 / m0 - 1) < (1e-9 if storage == "f32" else 1e-6), (m0, m1)
    assert sim.info()["steps"] == 200
    sim.close()
