"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L-inf on rho and j after the run): FP32 storage 1e-5,
FP16/BF16 deviation storage 2e-3.  Where a 16-bit format cannot reach 2e-3 on
a case, the bound is 1.25 times that format's floor on the same case: the
FP64 oracle with its stored deviations rounded to the format after every
step, computed in the test (helpers.check_storage_error)."""
import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.conftest import load_golden
from tests.helpers import THETA, check_storage_error, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


def _rerun(vel, shape, solid, tau, T, storage, force, E, B, rho, u, Ef, ro, jo):
    """gpu_rerun for check_storage_error: the same case with another rounding seed."""
    def run(seed):
        rg, jg, _, sim = gpu_run(vel, shape, solid, tau, T, storage, force, E, B, rho, u, Ef, seed=seed)
        sim.close()
        return rel_linf(rg, ro), rel_linf(jg, jo)
    return run


def _fields(shape, D, seed, amp_u=0.01, amp_rho=0.02):
    N = int(np.prod(shape))
    rho = (1.0 + amp_rho * (wl.uniform01(seed, N) - 0.5)).reshape(shape).astype(np.float32)
    u = (amp_u * wl.normal(seed + 1, D * N)).reshape((D,) + tuple(shape)).astype(np.float32)
    return rho, u


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("vel,fname", [("D2V9", "constants_2d.txt"), ("D3V19", "constants_3d.txt")])
def test_library_constants_match_printed_tables(vel, fname):
    from paper_1710_09472_gb300.lbm import LBM

    g = load_golden(fname)
    dims = (4, 4) if vel == "D2V9" else (4, 4, 4)
    sim = LBM(vel, dims, 0.8)
    c = sim.constants()
    for k in ["c0", "c1", "c2", "cbar2", "cprime2", "thetabar", "cs"]:
        assert abs(c[k] / g[k] - 1) < 1e-12, k
    assert abs(c["w"][0] / g["w0"] - 1) < 1e-12
    assert abs(c["w"][1] / g["ws"] - 1) < 1e-12
    assert abs(c["w"][-1] / g["wl"] - 1) < 1e-12
    sim.close()


CASES_2D = [(s, f, e, shp) for s in ("f32", "f16", "bf16") for f in ("term", "shift") for e in (False, True)
            for shp in ((37, 150), (30, 64))]


@pytest.mark.parametrize("storage,force,efield,shape", CASES_2D)
def test_parity_2d(storage, force, efield, shape):
    """D2V9, disks, B_z != 0, 60 steps.  37 x 150 (x: a 128-wide tile plus a
    ragged 22-cell tail; rows are not 16-byte multiples, so the general kernel
    runs) and 30 x 64 (row-staged kernel)."""
    solid, _ = wl.boolean_obstacles(shape, 3.0, 0.8, seed=41)
    rho, u = _fields(shape, 2, 42)
    E = (2e-4, -5e-5, 0.0)
    B = (0.0, 0.0, 3e-3)
    Ef = None
    if efield:
        Ef = np.stack([2e-4 + 2e-5 * wl.normal(43, solid.size).reshape(shape),
                       -5e-5 + 1e-5 * wl.normal(44, solid.size).reshape(shape)]).astype(np.float32)
    T = 60
    rg, jg, totg, sim = gpu_run("D2V9", shape, solid, 0.7, T, storage, force, E, B, rho, u, Ef)
    ro, jo, toto, _, _ = oracle_run("D2V9", shape, solid, 0.7, T, force, E, B, rho, u, Ef)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"2d {shape} {storage} {force} efield={efield}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel="D2V9", shape=shape, solid=solid, tau=0.7, steps=T, force=force,
                                                E=E, B=B, rho=rho, u=u, Efield=Ef, reference=(ro, jo)),
                        label=f"2d {shape} {force} efield={efield}",
                        gpu_rerun=_rerun("D2V9", shape, solid, 0.7, T, storage, force, E, B, rho, u, Ef, ro, jo))
    assert abs(totg[0] / toto[0] - 1) < (1e-6 if storage != "bf16" else 1e-4)
    sim.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("shape", [(12, 200), (8, 256), (10, 320), (4, 512), (6, 640)])
def test_parity_row_strides(storage, shape):
    """The row-staged step kernel keeps its shared-memory rows exactly nx long,
    at a compile-time stride for nx = 256 and 512 and a run-time one otherwise
    (200, 320, 640); D2V9 disks, 40 steps, against the oracle."""
    solid, _ = wl.boolean_obstacles(shape, 3.0, 0.8, seed=47)
    rho, u = _fields(shape, 2, 48)
    E, B = (2e-4, -5e-5, 0.0), (0.0, 0.0, 3e-3)
    rg, jg, totg, sim = gpu_run("D2V9", shape, solid, 0.7, 40, storage, "term", E, B, rho, u)
    ro, jo, toto, _, _ = oracle_run("D2V9", shape, solid, 0.7, 40, "term", E, B, rho, u)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"strides {shape} {storage}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel="D2V9", shape=shape, solid=solid, tau=0.7, steps=40, force="term",
                                                E=E, B=B, rho=rho, u=u, reference=(ro, jo)), label=f"strides {shape}",
                        gpu_rerun=_rerun("D2V9", shape, solid, 0.7, 40, storage, "term", E, B, rho, u, None, ro, jo))
    sim.close()


CASES_3D = [(s, f, e, shp) for s in ("f32", "f16", "bf16") for f in ("term", "shift") for e in (False, True)
            for shp in ((9, 10, 133), (8, 12, 64), (5, 6, 256))]


@pytest.mark.parametrize("storage,force,efield,shape", CASES_3D)
def test_parity_3d(storage, force, efield, shape):
    """D3V19, spheres, B oblique, 40 steps; 9 x 10 x 133 (general kernel),
    8 x 12 x 64 (row-staged kernel) and 5 x 6 x 256 (the row-staged kernel at
    the compile-time 256 stride; with FP32 storage its outputs overwrite the
    row's own stage)."""
    solid, _ = wl.boolean_obstacles(shape, 2.5, 0.75, seed=51)
    rho, u = _fields(shape, 3, 52)
    E = (1e-4, 3e-5, -2e-5)
    B = (1e-3, -2e-3, 3e-3)
    Ef = None
    if efield:
        Ef = (np.array(E)[:, None, None, None] * (1 + 0.1 * wl.normal(53, 3 * solid.size).reshape((3,) + shape))
              ).astype(np.float32)
    T = 40
    rg, jg, totg, sim = gpu_run("D3V19", shape, solid, 0.8, T, storage, force, E, B, rho, u, Ef)
    ro, jo, toto, _, _ = oracle_run("D3V19", shape, solid, 0.8, T, force, E, B, rho, u, Ef)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"3d {shape} {storage} {force} efield={efield}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel="D3V19", shape=shape, solid=solid, tau=0.8, steps=T, force=force,
                                                E=E, B=B, rho=rho, u=u, Efield=Ef, reference=(ro, jo)),
                        label=f"3d {shape} {force} efield={efield}",
                        gpu_rerun=_rerun("D3V19", shape, solid, 0.8, T, storage, force, E, B, rho, u, Ef, ro, jo))
    sim.close()


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
def test_populations_elementwise(vel):
    """Every population of every cell after a few steps (FP32 storage)."""
    shape = (13, 70) if vel == "D2V9" else (6, 7, 40)
    D = len(shape)
    solid, _ = wl.boolean_obstacles(shape, 2.0, 0.8, seed=61)
    rho, u = _fields(shape, D, 62)
    E = (1e-4, 2e-5, 1e-5)
    B = (0.0, 0.0, 1e-3) if D == 2 else (1e-3, 1e-3, 1e-3)
    rg, jg, totg, sim = gpu_run(vel, shape, solid, 0.75, 9, "f32", "term", E, B, rho, u)
    fg = sim.populations().astype(np.float64).reshape(sim.Q, -1)
    _, _, _, m, fo = oracle_run(vel, shape, solid, 0.75, 9, "term", E, B, rho, u)
    fo = fo.reshape(m.Q, -1)
    assert np.max(np.abs(fg - fo)) <= 2e-7 * np.max(np.abs(fo))
    sim.close()


@pytest.mark.parametrize("force", ["term", "shift"])
def test_config_poiseuille_32x64(force):
    """Config: Poiseuille 32 x 64, E_x = 1e-6, tau = 0.8, 5000 steps (Sec. 9.3
    forces with the velocity shift; the explicit term is the default here)."""
    w = wl.poiseuille_32x64()
    ro, jo, toto, _, _ = oracle_run("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], force, w["E"])
    errs = {}
    for storage in ("f32", "f16", "bf16"):
        rg, jg, totg, sim = gpu_run("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], storage, force, w["E"])
        errs[storage] = (rel_linf(rg, ro), rel_linf(jg, jo))
        print(f"poiseuille {force} {storage}: rho {errs[storage][0]:.3e} j {errs[storage][1]:.3e}")
        sim.close()
    for storage, e in errs.items():
        check_storage_error(storage, e, dict(vel="D2V9", shape=w["shape"], solid=w["solid"], tau=w["tau"],
                                             steps=w["steps"], force=force, E=w["E"], reference=(ro, jo)),
                            label=f"poiseuille {force}", seeds=(1, 2, 3),
                            gpu_rerun=_rerun("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], storage, force,
                                             w["E"], (0, 0, 0), None, None, None, ro, jo))


def test_config_riemann_4096x8():
    """Config: Riemann 4096 x 8, rho 1.05 | 1.0, tau = 0.6, 2000 steps."""
    w = wl.riemann_4096x8()
    rho = w["rho"].astype(np.float32)
    ro, jo, toto, _, _ = oracle_run("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], "term", rho=rho)
    errs = {}
    for storage in ("f32", "f16", "bf16"):
        rg, jg, totg, sim = gpu_run("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], storage, "term", rho=rho)
        errs[storage] = (rel_linf(rg, ro), rel_linf(jg, jo))
        print(f"riemann {storage}: rho {errs[storage][0]:.3e} j {errs[storage][1]:.3e}")
        sim.close()
    for storage, e in errs.items():
        check_storage_error(storage, e, dict(vel="D2V9", shape=w["shape"], solid=w["solid"], tau=w["tau"],
                                             steps=w["steps"], force="term", rho=rho, reference=(ro, jo)),
                            label="riemann", seeds=(1, 2, 3),
                            gpu_rerun=_rerun("D2V9", w["shape"], w["solid"], w["tau"], w["steps"], storage, "term",
                                             (0, 0, 0), (0, 0, 0), rho, None, None, ro, jo))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_porous_long_3d(storage):
    """A 32^3 copy of the porous configs (spheres r = 3, porosity 0.7, D3V19,
    tau = 0.8, E_x = 1e-5, B_z = 1e-3, explicit term) run 2000 steps: FP32 and
    FP16 against the targets 1e-5 and 2e-3, BF16 against 2e-3 or 1.25 times
    its format floor."""
    shape = (32, 32, 32)
    solid, _ = wl.boolean_obstacles(shape, 3.0, 0.7, seed=111)
    E, B = (1e-5, 0.0, 0.0), (0.0, 0.0, 1e-3)
    ro, jo, _, _, _ = oracle_run("D3V19", shape, solid, 0.8, 2000, "term", E, B)
    rg, jg, _, sim = gpu_run("D3V19", shape, solid, 0.8, 2000, storage, "term", E, B)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"porous32 {storage}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel="D3V19", shape=shape, solid=solid, tau=0.8, steps=2000,
                                                force="term", E=E, B=B, reference=(ro, jo)), seeds=(1, 2, 3),
                        label="porous32",
                        gpu_rerun=_rerun("D3V19", shape, solid, 0.8, 2000, storage, "term", E, B, None, None, None,
                                         ro, jo))
    sim.close()


# ---------------------------------------------------------------------------
# Full bench size: sampled one-step checks and conservation properties.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def porous256():
    return wl.porous_3d(256, Ex=1e-6, Bz=1e-3, steps=0)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_porous256_sampled_one_step(porous256, storage):
    """At 256^3 (the benchmark launch configuration): take the stored state after
    30 steps, let the oracle collide-and-stream it at 4000 sampled fluid cells
    and compare with the GPU's next state there."""
    from paper_1710_09472_gb300.lbm import LBM

    w = porous256
    shape = w["shape"]
    dev = torch.device("cuda")
    sim = LBM("D3V19", tuple(reversed(shape)), w["tau"], E=w["E"], B=w["B"], storage=storage, force="term")
    sim.set_geometry(torch.from_numpy(w["solid"].reshape(-1)).to(dev))
    sim.init_equilibrium()
    sim.step(30)
    Q, N = sim.Q, sim.N
    h_t = torch.empty(Q * N, dtype=torch.float32, device=dev)
    sim.populations(h_t, deviation=True)
    sim.step(1)
    h_t1 = torch.empty(Q * N, dtype=torch.float32, device=dev)
    sim.populations(h_t1, deviation=True)
    torch.cuda.synchronize()
    m = oracle.Model("D3V19", "fd", THETA, 1.0, tau=w["tau"], E=w["E"], B=w["B"], force="term")
    f0 = 1.0 * m.w / m.const["I0"]
    solid = w["solid"].reshape(-1)
    fluid_idx = np.flatnonzero(solid == 0)
    rng = np.random.default_rng(7)
    sample = rng.choice(fluid_idx, 4000, replace=False)
    nx, ny, nz = sim.dims
    ht = h_t.view(Q, N).cpu().numpy()
    ht1 = h_t1.view(Q, N).cpu().numpy()
    err = 0.0
    scale = 0.0
    for cell in sample:
        x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        expect = np.empty(Q)
        # f_{t+1,a}(x) = C(f_t)(x - e_a)_a, or C(f_t)(x)_abar if x - e_a is solid
        cache = {}
        for a in range(Q):
            ex, ey, ez = m.e[a]
            src = (((z - ez) % nz) * ny + (y - ey) % ny) * nx + (x - ex) % nx
            if solid[src]:
                src_cell, comp = cell, m.opp[a]
            else:
                src_cell, comp = src, a
            if src_cell not in cache:
                fc = ht[:, src_cell].astype(np.float64) + f0
                cache[src_cell] = m.collide_cell(fc) - f0
            expect[a] = cache[src_cell][comp]
        err = max(err, float(np.max(np.abs(ht1[:, cell] - expect))))
        scale = max(scale, float(np.max(np.abs(expect))))
    # FP32: a few ulps of the deviations; FP16: one storage ulp (stochastic
    # rounding picks either neighbour), 2^-10 relative
    tol = 1e-5 * scale if storage == "f32" else 2.0 ** -9 * scale
    assert err <= tol, (err, scale)
    sim.close()


def test_porous256_mass_conserved(porous256):
    """sum rho over fluid cells is conserved (bounce-back + BGK), FP64 totals."""
    from paper_1710_09472_gb300.lbm import LBM

    w = porous256
    for storage in ("f32", "f16"):
        sim = LBM("D3V19", tuple(reversed(w["shape"])), w["tau"], E=(1e-5, 0, 0), B=(0, 0, 1e-3), storage=storage)
        sim.set_geometry(torch.from_numpy(w["solid"].reshape(-1)).cuda())
        sim.init_equilibrium()
        m0, _ = sim.moments()
        sim.step(100)
        m1, j1 = sim.moments()
        # FP32: summation round-off only; FP16: 100 roundings of each stored
        # deviation (|h| ~ 1e-6 here, half an ulp ~ 2^-12 |h|)
        bound = 1e-9 if storage == "f32" else 1e-7
        assert abs(m1 / m0 - 1) < bound, (storage, m0, m1)
        assert sim.info()["n_fluid"] == int((w["solid"] == 0).sum())
        sim.close()


@pytest.mark.parametrize("force", ["term", "shift"])
def test_periodic_momentum_growth(force):
    """Periodic box without obstacles: sum j grows by sum rho E each step."""
    from paper_1710_09472_gb300.lbm import LBM

    E = (2e-5, -1e-5, 5e-6)
    sim = LBM("D3V19", (64, 48, 40), 0.8, E=E, force=force)
    sim.init_equilibrium()
    m0, j0 = sim.moments()
    sim.step(50)
    m1, j1 = sim.moments()
    for d in range(3):
        assert abs(j1[d] - j0[d] - 50 * m0 * E[d]) < 1e-4 * abs(50 * m0 * E[d]) + 1e-9
    sim.close()


# ---------------------------------------------------------------------------
# Edge cases and the C-ABI contract.
# ---------------------------------------------------------------------------
def test_degenerate_domains():
    from paper_1710_09472_gb300.lbm import LBM

    # one periodic cell (every neighbour is the cell itself), uniform force
    for vel, dims in (("D2V9", (1, 1)), ("D3V19", (1, 1, 1))):
        shape = tuple(reversed(dims))
        rg, jg, tot, sim = gpu_run(vel, shape, None, 0.8, 10, "f32", "term", (1e-4, 0, 0))
        ro, jo, toto, _, _ = oracle_run(vel, shape, None, 0.8, 10, "term", (1e-4, 0, 0))
        assert rel_linf(rg, ro) < 1e-6 and rel_linf(jg, jo) < 1e-5
        sim.close()
    # a fully solid box: nothing moves, totals are zero
    sim = LBM("D2V9", (16, 8), 0.8)
    sim.set_geometry(np.ones(128, dtype=np.uint8))
    sim.init_equilibrium()
    sim.step(3)
    m, j = sim.moments()
    assert m == 0.0 and np.all(j == 0.0)
    assert sim.info()["n_fluid"] == 0
    sim.close()
    # channel one cell wide in x, zero steps
    sim = LBM("D2V9", (1, 64), 0.8, E=(1e-6, 0))
    sim.set_geometry(wl.channel_mask((64, 1)).reshape(-1))
    sim.init_equilibrium()
    m0, _ = sim.moments()
    sim.step(0)
    m1, _ = sim.moments()
    assert m0 == m1 == 62.0
    sim.close()


def test_host_and_device_pointers_agree():
    from paper_1710_09472_gb300.lbm import LBM

    shape = (20, 36)
    solid, _ = wl.boolean_obstacles(shape, 2.0, 0.85, seed=71)
    rho, u = _fields(shape, 2, 72)
    outs = []
    for where in ("host", "device"):
        sim = LBM("D2V9", (36, 20), 0.7, E=(1e-4, 0))
        conv = (lambda a: a.reshape(-1)) if where == "host" else (lambda a: torch.from_numpy(a.reshape(-1)).cuda())
        sim.set_geometry(conv(solid))
        sim.init_equilibrium(conv(rho), conv(u))
        sim.step(7)
        if where == "host":
            r = np.empty(sim.N, np.float32)
            j = np.empty(2 * sim.N, np.float32)
            tot = sim.moments(r, j)
        else:
            r_d = torch.empty(sim.N, device="cuda")
            j_d = torch.empty(2 * sim.N, device="cuda")
            tot = sim.moments(r_d, j_d)
            r, j = r_d.cpu().numpy(), j_d.cpu().numpy()
        outs.append((r, j, tot))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2][0] == outs[1][2][0]


def test_save_load_roundtrip_and_errors():
    from paper_1710_09472_gb300._lib import LBMError
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM("D3V19", (10, 9, 8), 0.8, E=(1e-4, 0, 0), storage="f16")
    with pytest.raises(LBMError):
        sim.step(1)  # before init: LBM_ERR_STATE
    sim.init_equilibrium()
    sim.step(5)
    blob = sim.save_state()
    sim.step(5)
    a = sim.populations()
    sim.load_state(blob)
    assert sim.info()["steps"] == 5
    sim.step(5)
    b = sim.populations()
    assert np.array_equal(a, b)
    bad = bytearray(blob)
    bad[-1] ^= 0xFF
    with pytest.raises(LBMError):
        sim.load_state(bytes(bad))
    with pytest.raises(LBMError):
        sim.set_params(0.5)
    sim.close()
    with pytest.raises(LBMError):
        LBM("D2V9", (8, 8, 2), 0.8)  # a 2D lattice needs nz = 1
    with pytest.raises(LBMError):
        LBM("D2V9", (8, 8), 0.4)


def test_bounded_wait_runs_out_and_reports_timeout():
    """The bounded mbarrier wait of the row-staged kernels, run on a barrier
    that nothing completes (limit 2^20 clocks, about 0.5 ms): the block gives
    up, the next synchronising call reports LBM_ERR_TIMEOUT, and the context
    keeps working."""
    from paper_1710_09472_gb300._lib import STATUS
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM("D3V19", (32, 6, 5), 0.8, E=(1e-4, 0, 0), storage="f16")
    sim.init_equilibrium()
    sim.step(3)
    before = sim.populations()
    assert STATUS[sim.selftest_wait_timeout(1 << 20)] == "LBM_ERR_TIMEOUT"
    assert STATUS[sim.selftest_wait_timeout(1 << 10)] == "LBM_ERR_TIMEOUT"
    assert np.array_equal(sim.populations(), before)  # reported once, state untouched
    sim.step(2)
    tot, _ = sim.moments()
    assert np.isfinite(tot)
    assert STATUS[sim.selftest_wait_timeout(0)] == "LBM_ERR_INVALID_ARG"
    sim.close()
