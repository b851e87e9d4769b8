"""lbm_moment_totals_static, the entry point that allocates nothing, called
through the C ABI.  It is for callers that cannot call cudaMalloc where they
read the totals (an application whose device memory is all reserved up front
by its own pool, or a loop in which allocation calls are forbidden), so its
per-block partial sums live in a fixed device array of the library.

The checks: its totals equal those of lbm_moments on two calls in a row (the
array keeps the previous call's contents), they match the FP64 oracle's
totals, grids with several x-blocks per row index the partials correctly, and
a grid needing more partials than the array holds is rejected with
INVALID_ARG and a message.  The file is named so that pytest collects it last:
a run that stops at the first failure has then run every other test.  The
tests create their own contexts and pass alone or after the others."""
import numpy as np
import pytest

from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import oracle_run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


def _static_vs_moments(sim, steps_each, calls=2):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    got = []
    for _ in range(calls):
        sim.step(steps_each)
        ref_rho, ref_j = sim.moments()
        sim.moment_totals_static(out)
        torch.cuda.synchronize()
        g = out.cpu().numpy().copy()
        assert abs(g[0] / ref_rho - 1) < 1e-12
        scale = max(np.abs(ref_j).max(), 1e-300)
        assert np.max(np.abs(g[1:] - ref_j)) <= 1e-12 * scale
        got.append(g)
    return got


@pytest.mark.parametrize("shape", [(24, 30, 64), (6, 5, 300)])
def test_static_totals_match_lbm_moments_twice(shape):
    """D3V19 spheres, FP16 storage; 64 wide (one 128-cell block per row) and
    300 wide (three x-blocks per row, so the partial index runs over x-blocks
    too)."""
    from paper_1710_09472_gb300.lbm import LBM

    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.75, seed=101)
    sim = LBM("D3V19", tuple(reversed(shape)), 0.8, E=(1e-4, 2e-5, 0.0), B=(0.0, 0.0, 1e-3), storage="f16")
    sim.set_geometry(torch.from_numpy(mask.reshape(-1)).cuda())
    sim.init_equilibrium()
    _static_vs_moments(sim, 7)
    sim.close()


def test_static_totals_match_oracle():
    """FP32 storage, 300-wide rows, 12 steps: the static totals against the
    FP64 oracle's totals over the fluid cells (sum rho to 1e-7 relative, the
    current to 1e-5 of its largest component)."""
    from paper_1710_09472_gb300.lbm import LBM

    shape = (6, 5, 300)
    mask, _ = wl.boolean_obstacles(shape, 2.5, 0.75, seed=103)
    E, B = (2e-4, -3e-5, 1e-5), (1e-3, 0.0, 2e-3)
    sim = LBM("D3V19", tuple(reversed(shape)), 0.8, E=E, B=B, storage="f32", force="term")
    sim.set_geometry(torch.from_numpy(mask.reshape(-1)).cuda())
    sim.init_equilibrium()
    got = _static_vs_moments(sim, 6)
    _, _, tot, _, _ = oracle_run("D3V19", shape, mask, 0.8, 12, "term", E, B)
    g = got[-1]
    assert abs(g[0] / tot[0] - 1) < 1e-7, (g[0], tot[0])
    assert np.max(np.abs(g[1:] - tot[1:])) <= 1e-5 * np.max(np.abs(tot[1:])), (g, tot)
    sim.close()


def test_static_totals_capacity():
    """ny * nz * ceil(nx / 128) partials: 262144 fit (a 1 x 262144 D2V9 box),
    262145 are rejected with INVALID_ARG and a message naming the limit."""
    from paper_1710_09472_gb300._lib import LBMError
    from paper_1710_09472_gb300.lbm import LBM

    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    sim = LBM("D2V9", (1, 262144), 0.8, E=(1e-5, 0.0))
    sim.init_equilibrium()
    sim.step(2)
    ref_rho, _ = sim.moments()
    sim.moment_totals_static(out)
    torch.cuda.synchronize()
    assert abs(float(out[0]) / ref_rho - 1) < 1e-12
    sim.close()
    sim = LBM("D2V9", (1, 262145), 0.8, E=(1e-5, 0.0))
    sim.init_equilibrium()
    with pytest.raises(LBMError) as ei:
        sim.moment_totals_static(out)
    assert "LBM_ERR_INVALID_ARG" in str(ei.value) and "262144" in str(ei.value)
    sim.close()
