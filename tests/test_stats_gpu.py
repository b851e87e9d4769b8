"""Other weights through the same kernels: Bose-Einstein and Maxwell-Boltzmann
(Sec. 3, the weight omega of Eq. i2n-cont2; MB with theta = 1 is the Hermite
weight, so D2V9/D3V19 become the textbook lattices).  Only the host constants
change; the GPU path is compared with the FP64 oracle built for the same
weight."""
import numpy as np
import pytest

from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import check_storage_error, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


STATS = [("mb", 1.0, 0.0), ("be", 0.5, -0.2)]


@pytest.mark.parametrize("stat,theta,mu", STATS)
@pytest.mark.parametrize("vel,shape", [("D2V9", (48, 64)), ("D3V19", (12, 16, 32))])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_other_weights_match_oracle(stat, theta, mu, vel, shape, storage):
    import oracle
    from paper_1710_09472_gb300.lbm import LBM

    solid, _ = wl.boolean_obstacles(shape, 2.5, 0.8, seed=121)
    E = (2e-4, -1e-4, 5e-5) if vel == "D3V19" else (2e-4, -1e-4, 0.0)
    B = (1e-2, 0.0, 2e-2) if vel == "D3V19" else (0.0, 0.0, 2e-2)
    tau, steps = 0.75, 300
    N = int(np.prod(shape))
    rho0 = (1.0 + 0.01 * wl.uniform01(122, N)).reshape(shape)
    m = oracle.Model(vel, stat, theta, mu, tau=tau, E=E, B=B, force="term")
    f = m.init_equilibrium(shape, solid, rho0)
    m.step(shape, solid, f, steps)
    ro, jo, _ = m.moments(shape, solid, f)

    sim = LBM(vel, tuple(reversed(shape)), tau, E=E, B=B, storage=storage, force="term", stat=stat, theta=theta,
              mu=mu)
    dev = torch.device("cuda")
    sim.set_geometry(torch.from_numpy(solid.reshape(-1)).to(dev))
    sim.init_equilibrium(torch.from_numpy(rho0.reshape(-1).astype(np.float32)).to(dev))
    sim.step(steps)
    rho = torch.empty(N, device=dev)
    j = torch.empty(sim.D * N, device=dev)
    sim.moments(rho, j)
    er = rel_linf(rho.cpu().numpy().reshape(shape), ro)
    ej = rel_linf(j.cpu().numpy().reshape((sim.D,) + shape), jo)
    print(f"{stat} {vel} {storage}: rho {er:.3e} j {ej:.3e}")
    check_storage_error(storage, (er, ej), dict(vel=vel, shape=shape, solid=solid, tau=tau, steps=steps, force="term",
                                                E=E, B=B, rho=rho0, reference=(ro, jo), stat=stat, theta=theta,
                                                mu=mu), label=f"{stat} {vel}")
    sim.close()
