"""GPU parity of the local chemical-potential model (lbm_set_local_mu): the
EDF of Sec. 9.1, Eq. feq-exp-2nd-order-eq, with each cell's thetabar = I_2/I_0
at the chemical potential of its own density (Eq. rho-def-eq), against the
FP64 oracle's Model.step_local_mu / collide_cell_thetabar, and its adjoint
against Model.adjoint_local_mu.

Tolerances as for the default model: relative L-inf on rho and j, FP32
storage 1e-5, FP16 deviation storage 2e-3."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import TOL, deviations_on_device, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


# FD weight at theta = 0.5, mu = 0: the local thetabar raises the sound speed
# by 8% over the constant-thetabar model (0.649 against 0.601 lattice units);
# more degenerate 2D weights push it to the lattice limit of 1 (theta = 1/270:
# exactly 1.000), where the BGK step is unstable.
THETA, MU = 0.5, 0.0
SHAPE = (40, 64)


def _case(seed=7):
    yy, xx = np.mgrid[0:SHAPE[0], 0:SHAPE[1]]
    solid = ((((xx - 20) ** 2 + (yy - 14) ** 2) < 36) | (((xx - 45) ** 2 + (yy - 27) ** 2) < 25)).astype(np.uint8)
    rho = 1.0 + 0.02 * (wl.uniform01(seed, SHAPE[0] * SHAPE[1]).reshape(SHAPE) - 0.5)
    return solid, rho


def _gpu(vel, shape, solid, rho, steps, storage="f32", force="term", E=(2e-4, 0.0, 0.0), B=(0.0, 0.0, 5e-3),
         stat="fd", theta=THETA, mu=MU, local=True, tau=0.8):
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM(vel, tuple(reversed(shape)), tau, E=E, B=B, storage=storage, force=force, stat=stat, theta=theta,
              mu=mu)
    dev = torch.device("cuda")
    sim.set_geometry(torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)).to(dev))
    if local:
        sim.set_local_mu(True)
    sim.init_equilibrium(torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32).reshape(-1)).to(dev))
    sim.step(steps)
    r = torch.empty(sim.N, device=dev)
    j = torch.empty(sim.D * sim.N, device=dev)
    tot = sim.moments(r, j)
    torch.cuda.synchronize()
    return r.cpu().numpy().reshape(shape), j.cpu().numpy().reshape((sim.D,) + tuple(shape)), tot, sim


def _oracle(vel, shape, solid, rho, steps, force="term", E=(2e-4, 0.0, 0.0), B=(0.0, 0.0, 5e-3), stat="fd",
            theta=THETA, mu=MU, local=True, tau=0.8):
    m = oracle.Model(vel, stat, theta, mu, tau=tau, E=E, B=B, force=force)
    f = m.init_equilibrium(shape, solid, np.asarray(rho, dtype=np.float32).astype(np.float64))
    if local:
        m.step_local_mu(shape, solid, f, steps, rho_ref=1.0)
    else:
        m.step(shape, solid, f, steps)
    r, j, tot = m.moments(shape, solid, f)
    return r, j, tot, m


@pytest.mark.parametrize("force", ["term", "shift"])
def test_local_mu_parity_2d_f32(force):
    """D2V9 with two obstacles, E and B, 2% density noise, 300 steps, FP32
    storage: rho and j within 1e-5 of the oracle; the constant-thetabar model
    differs from both by far more (the switch acts)."""
    solid, rho = _case()
    rg, jg, tg, sim = _gpu("D2V9", SHAPE, solid, rho, 300, force=force)
    sim.close()
    ro, jo, to, _ = _oracle("D2V9", SHAPE, solid, rho, 300, force=force)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    rb, jb, _, _ = _oracle("D2V9", SHAPE, solid, rho, 300, force=force, local=False)
    gap = rel_linf(jb, jo)
    print(f"local mu 2D {force}: rho {er:.2e} j {ej:.2e}; constant-thetabar model differs by {gap:.2e}")
    assert er <= TOL["f32"] and ej <= TOL["f32"], (er, ej)
    assert gap > 100 * TOL["f32"]
    assert abs(tg[0] / to[0] - 1) < 1e-6


def test_local_mu_parity_2d_f16():
    """The same case in FP16 deviation storage (200 steps): within 2e-3."""
    solid, rho = _case(11)
    rg, jg, _, sim = _gpu("D2V9", SHAPE, solid, rho, 200, storage="f16")
    sim.close()
    ro, jo, _, _ = _oracle("D2V9", SHAPE, solid, rho, 200)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"local mu 2D f16: rho {er:.2e} j {ej:.2e}")
    assert er <= TOL["f16"] and ej <= TOL["f16"], (er, ej)


def test_local_mu_mb_equals_default_model():
    """With the MB weight thetabar does not depend on mu: the local model (its
    own row-staged instantiation, a zero table) equals the default model to
    FP32 rounding."""
    solid, rho = _case(3)
    args = dict(stat="mb", theta=1.0, mu=0.0)
    r1, j1, _, s1 = _gpu("D2V9", SHAPE, solid, rho, 100, **args)
    r2, j2, _, s2 = _gpu("D2V9", SHAPE, solid, rho, 100, local=False, **args)
    s1.close()
    s2.close()
    assert rel_linf(r1, r2) < 1e-6 and rel_linf(j1, j2) < 1e-5


@pytest.mark.parametrize("dims", [(24, 20, 16), (64, 12, 10)])
def test_local_mu_3d_sampled_step(dims):
    """D3V19 at the paper's copper values (theta = 1/270, mu = 1: the
    Sommerfeld branch of the device table) on a porous box (nx = 24: the
    general kernel; nx = 64: the row-staged kernel's local-mu instantiation):
    after 20 GPU steps of the local model, one more GPU step against the
    oracle's collision with thetabar from the cell-by-cell FD route
    (mu_of_density, then I_2/I_0), at sampled fluid cells and every
    direction."""
    from paper_1710_09472_gb300.lbm import LBM

    theta, mu = 1.0 / 270.0, 1.0
    nx, ny, nz = dims
    mask, _ = wl.boolean_obstacles((nz, ny, nx), 3.0, 0.8, 9)
    solid_flat = mask.reshape(-1).astype(np.uint8)
    rho = 1.0 + 2e-3 * (wl.uniform01(5, nx * ny * nz) - 0.5)
    E = (3e-5, 1e-5, 0.0)
    B = (0.0, 2e-3, 1e-2)
    sim = LBM("D3V19", dims, 0.8, E=E, B=B, storage="f32", force="term", theta=theta, mu=mu)
    dev = torch.device("cuda")
    sim.set_geometry(torch.from_numpy(solid_flat).to(dev))
    sim.set_local_mu(True)
    sim.init_equilibrium(torch.from_numpy(rho.astype(np.float32)).to(dev))
    sim.step(20)
    h_t = deviations_on_device(sim).clone()
    sim.step(1)
    h_t1 = deviations_on_device(sim)
    m = oracle.Model("D3V19", "fd", theta, mu, tau=0.8, E=E, B=B, force="term")
    f0 = m.w / m.const["I0"]
    fluid = np.flatnonzero(solid_flat == 0)
    cells = fluid[(wl.uniform01(13, 8) * fluid.size).astype(np.int64)]
    worst, scale = 0.0, 0.0
    for cell in cells:
        x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        srcs = []
        for a in range(m.Q):
            ex, ey, ez = m.e[a]
            src = (((z - ez) % nz) * ny + (y - ey) % ny) * nx + (x - ex) % nx
            srcs.append((cell, m.opp[a]) if solid_flat[src] else (src, a))
        after = h_t1[:, int(cell)].cpu().numpy().astype(np.float64)
        expect = np.empty(m.Q)
        cache = {}
        for a, (sc, comp) in enumerate(srcs):
            if sc not in cache:
                fc = h_t[:, int(sc)].cpu().numpy().astype(np.float64) + f0
                thb = m.local_thetabar(np.array([fc.sum()]), rho_ref=1.0)[0]
                cache[sc] = m.collide_cell_thetabar(fc, thb) - f0
            expect[a] = cache[sc][comp]
        worst = max(worst, float(np.max(np.abs(after - expect))))
        scale = max(scale, float(np.max(np.abs(expect))))
    sim.close()
    print(f"local mu 3D sampled step: max |err| {worst:.3e} of max |h| {scale:.3e}")
    assert worst <= 1e-5 * scale


def test_local_mu_sound_speed_gpu():
    """A standing density wave (D2V9 row of 64 cells, FP32, FD theta = 0.5,
    mu = 0) runs at c_s sqrt(thetabar + rho thetabar'(rho)), the sound speed of
    the FD equation of state p = rho thetabar(rho), within 2e-3."""
    from paper_1710_09472_gb300.lbm import LBM

    nx = 64
    m = oracle.Model("D2V9", "fd", THETA, MU)
    h = 1e-6
    dth = (m.local_thetabar(np.array([1 + h]), 1.0)[0] - m.local_thetabar(np.array([1 - h]), 1.0)[0]) / (2 * h)
    want = m.const["cs"] * math.sqrt(m.const["thetabar"] + dth)
    sim = LBM("D2V9", (nx, 1), 0.6, storage="f32", theta=THETA, mu=MU)
    sim.set_local_mu(True)
    x = np.arange(nx)
    dev = torch.device("cuda")
    sim.init_equilibrium(torch.from_numpy((1 + 1e-5 * np.cos(2 * np.pi * x / nx)).astype(np.float32)).to(dev))
    j = torch.empty(2 * nx, device=dev)
    probe = []
    for _ in range(500):
        sim.step(1)
        sim.moments(None, j, totals=False)
        probe.append(float(j[nx // 4]))
    sim.close()
    probe = np.array(probe)
    s = np.sign(probe)
    cross = np.flatnonzero(s[1:] != s[:-1])
    tc = np.array([c + probe[c] / (probe[c] - probe[c + 1]) for c in cross])
    c = nx / (2 * float(np.mean(np.diff(tc))))
    print(f"local mu sound speed {c:.6f} vs {want:.6f} (constant thetabar {m.const['cs'] * math.sqrt(m.const['thetabar']):.6f})")
    assert abs(c / want - 1) < 2e-3


@pytest.mark.parametrize("force", ["term", "shift"])
@pytest.mark.parametrize("nx", [40, 38])
def test_local_mu_adjoint_matches_oracle(force, nx):
    """lbm_adjoint of the local model (row-staged reverse kernel for nx = 40,
    the general one for nx = 38) against the oracle's reverse sweep of the
    same model (pinned to finite differences on the CPU): per-cell dL/dE,
    dL/df_0, dL/dB_z and dL/dtau to 1e-4, the loss to 1e-5."""
    from paper_1710_09472_gb300.lbm import LBM

    shape = (14, nx)
    mask, _ = wl.boolean_obstacles(shape, 2.5, 0.8, seed=81)
    N = mask.size
    B = (0.0, 0.0, 2e-2)
    Ef = np.zeros((2,) + shape, dtype=np.float32)
    Ef[0] = (1e-3 + 2e-4 * wl.normal(83, N)).reshape(shape)
    Ef[1] = (3e-4 * wl.normal(84, N)).reshape(shape)
    rho0 = (1.0 + 0.02 * wl.uniform01(85, N)).reshape(shape).astype(np.float32)
    u0 = (0.01 * wl.normal(86, 2 * N)).reshape((2,) + shape).astype(np.float32)
    wr = wl.normal(87, N).reshape(shape).astype(np.float32)
    wj = wl.normal(88, 2 * N).reshape((2,) + shape).astype(np.float32)
    tau, T, tb = 0.75, 14, 6
    sim = LBM("D2V9", (nx, 14), tau, B=B, storage="f32", force=force, theta=THETA, mu=MU)
    sim.set_geometry(mask.reshape(-1))
    sim.set_E_field(torch.from_numpy(Ef.reshape(-1)).cuda())
    sim.set_local_mu(True)
    sim.init_equilibrium(torch.from_numpy(rho0.reshape(-1)).cuda(), torch.from_numpy(u0.reshape(-1)).cuda())
    dE = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(9 * N, dtype=torch.float32, device="cuda")
    res = sim.adjoint(tb, T, torch.from_numpy(wr.reshape(-1)).cuda(), torch.from_numpy(wj.reshape(-1)).cuda(),
                      checkpoint_every=4, dL_dE=dE, dL_df0=lam0)
    sim.close()
    m = oracle.Model("D2V9", "fd", THETA, MU, tau=tau, B=B, force=force)
    E64 = Ef.astype(np.float64)
    f = m.init_equilibrium(shape, mask, rho0.astype(np.float64), u0.astype(np.float64))
    states = np.empty((T + 1, f.size))
    states[0] = f
    for t in range(T):
        m.step_local_mu(shape, mask, f, 1, E64, rho_ref=1.0)
        states[t + 1] = f
    ref = m.adjoint_local_mu(shape, mask, states, tb, T, wr.astype(np.float64), wj.astype(np.float64), E64,
                             rho_ref=1.0)
    eg = rel_linf(dE.cpu().numpy().reshape(ref["gE"].shape), ref["gE"])
    el = rel_linf(lam0.cpu().numpy(), ref["lam0"])
    print(f"local mu adjoint nx={nx} {force}: dL/dE {eg:.2e} dL/df0 {el:.2e} dL/dtau {res['dL_dtau']:.6e} "
          f"vs {ref['gtau']:.6e}")
    assert abs(res["loss"] / ref["loss"] - 1) < 1e-5
    assert eg < 1e-4 and el < 1e-4, (eg, el)
    assert abs(res["dL_dB"][2] - ref["gB"][2]) < 1e-4 * max(abs(ref["gB"][2]), 1e-2 * np.abs(ref["gB"]).max())
    assert abs(res["dL_dtau"] / ref["gtau"] - 1) < 1e-4


def test_local_mu_errors():
    from paper_1710_09472_gb300._lib import LBMError
    from paper_1710_09472_gb300.lbm import LBM

    for vel, dims, stat, theta, mu in (("D3V27", (8, 8, 8), "mb", 1.0, 0.0), ("D2V9", (16, 8), "be", 0.5, -0.3)):
        sim = LBM(vel, dims, 0.8, stat=stat, theta=theta, mu=mu)
        with pytest.raises(LBMError):
            sim.set_local_mu(True)
        sim.close()
    sim = LBM("D2V9", (16, 8), 0.8, theta=THETA, mu=MU)
    sim.set_local_mu(True)
    sim.set_local_mu(True)  # enabling twice keeps the table
    sim.init_equilibrium()
    sim.step(2)
    sim.set_local_mu(False)
    sim.step(2)
    sim.close()
