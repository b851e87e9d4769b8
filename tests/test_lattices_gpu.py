"""D3V27 and D1V3 through the same kernels (Table lattices-tab, Sec. 8.1):
constants, 40-step parity of the step kernels and the reverse step, each
against the FP64 oracle.  Needs a GPU."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import THETA, check_storage_error, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


def _case(vel, shape, seed):
    """Solid mask (spheres in 3D, isolated solid cells in 1D), fields and forces."""
    N = int(np.prod(shape))
    if vel == "D1V3":
        solid = (wl.uniform01(seed, N) < 0.08).reshape(shape).astype(np.uint8)
        E, B = (2e-4, 0.0, 0.0), (0.0, 0.0, 0.0)
    else:
        solid, _ = wl.boolean_obstacles(shape, 2.5, 0.75, seed=seed)
        E, B = (1e-4, 3e-5, -2e-5), (1e-3, -2e-3, 3e-3)
    D = len(shape)
    rho = (1.0 + 0.02 * (wl.uniform01(seed + 1, N) - 0.5)).reshape(shape).astype(np.float32)
    u = (0.01 * wl.normal(seed + 2, D * N)).reshape((D,) + tuple(shape)).astype(np.float32)
    return solid, E, B, rho, u


@pytest.mark.parametrize("vel,dims", [("D3V27", (4, 4, 4)), ("D1V3", (16,))])
def test_constants_match_oracle(vel, dims):
    """Weights and c_s of the library (FP64 host constants) equal the oracle's."""
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM(vel, dims, 0.8)
    c = sim.constants()
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=0.8)
    assert sim.Q == m.Q
    assert abs(c["cs"] / m.const["cs"] - 1) < 1e-12
    np.testing.assert_allclose(c["w"], m.w, rtol=1e-12, atol=0)
    sim.close()


# staged: nx a multiple of 16 bytes per row; general: a ragged nx
SHAPES = {("D3V27", "staged"): (8, 10, 64), ("D3V27", "general"): (6, 7, 35),
          ("D1V3", "staged"): (256,), ("D1V3", "general"): (250,)}


@pytest.mark.parametrize("vel", ["D3V27", "D1V3"])
@pytest.mark.parametrize("layout", ["staged", "general"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("force", ["term", "shift"])
def test_step_parity(vel, layout, storage, force):
    shape = SHAPES[(vel, layout)]
    solid, E, B, rho, u = _case(vel, shape, 61)
    rg, jg, totg, sim = gpu_run(vel, shape, solid, 0.8, 40, storage, force, E, B, rho, u)
    ro, jo, toto, _, _ = oracle_run(vel, shape, solid, 0.8, 40, force, E, B, rho, u)
    er, ej = rel_linf(rg, ro), rel_linf(jg, jo)
    print(f"{vel} {layout} {storage} {force}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel=vel, shape=shape, solid=solid, tau=0.8, steps=40, force=force,
                                                E=E, B=B, rho=rho, u=u, reference=(ro, jo)),
                        label=f"{vel} {layout} {force}")
    # FP32 conserves the total to rounding; a 16-bit store rounds each value by up
    # to half an ulp of 2^12 h, about 1e-6 of the total over these few cells
    assert abs(totg[0] / toto[0] - 1) < (1e-6 if storage == "f32" else 1e-5)
    sim.close()


@pytest.mark.parametrize("vel,shape", [("D3V27", (6, 7, 36)), ("D3V27", (6, 7, 35)), ("D1V3", (128,))])
@pytest.mark.parametrize("force", ["term", "shift"])
def test_adjoint_matches_oracle(vel, shape, force):
    import torch

    from paper_1710_09472_gb300.lbm import LBM

    solid, E, B, rho0, u0 = _case(vel, shape, 71)
    D, N = len(shape), int(np.prod(shape))
    Ef = np.zeros((D,) + shape, dtype=np.float32)
    Ef[0] = (1e-3 + 2e-4 * wl.normal(73, N)).reshape(shape)
    if D > 1:
        Ef[1] = (3e-4 * wl.normal(74, N)).reshape(shape)
    wr = wl.normal(75, N).reshape(shape).astype(np.float32)
    wj = wl.normal(76, D * N).reshape((D,) + shape).astype(np.float32)
    tau, T, tb = 0.75, 12, 5
    sim = LBM(vel, tuple(reversed(shape)), tau, B=B, storage="f32", force=force)
    sim.set_geometry(torch.from_numpy(solid.reshape(-1)).cuda())
    sim.set_E_field(torch.from_numpy(Ef.reshape(-1)).cuda())
    sim.init_equilibrium(torch.from_numpy(rho0.reshape(-1)).cuda(), torch.from_numpy(u0.reshape(-1)).cuda())
    dE = torch.empty(D * N, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(sim.Q * N, dtype=torch.float32, device="cuda")
    res = sim.adjoint(tb, T, torch.from_numpy(wr.reshape(-1)).cuda(), torch.from_numpy(wj.reshape(-1)).cuda(),
                      checkpoint_every=4, dL_dE=dE, dL_df0=lam0)
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, B=B, force=force)
    f0 = m.init_equilibrium(shape, solid, rho0.astype(np.float64), u0.astype(np.float64))
    states = m.trajectory(shape, solid, f0, T, Ef.astype(np.float64))
    ref = m.adjoint(shape, solid, states, tb, T, wr.astype(np.float64), wj.astype(np.float64),
                    Ef.astype(np.float64))
    assert abs(res["loss"] / ref["loss"] - 1) < 1e-5
    gE = dE.cpu().numpy().reshape(ref["gE"].shape)
    assert rel_linf(gE, ref["gE"]) < 1e-4, rel_linf(gE, ref["gE"])
    assert rel_linf(lam0.cpu().numpy(), ref["lam0"]) < 1e-4
    assert abs(res["dL_dtau"] / ref["gtau"] - 1) < 1e-4
    if vel == "D3V27":
        for c in range(3):
            assert abs(res["dL_dB"][c] - ref["gB"][c]) < 1e-4 * max(abs(ref["gB"][c]), 1e-2 * np.abs(ref["gB"]).max())
    sim.close()
