"""lbm_moment_totals_static: the allocation-free totals entry point, called
through the C ABI, must agree with the totals of lbm_moments on two calls in
a row (this file is collected last on purpose)."""
import numpy as np
import pytest

from paper_1710_09472_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_totals_match_lbm_moments_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build
    from paper_1710_09472_gb300.lbm import LBM

    build()
    shape = (24, 30, 64)
    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.75, seed=101)
    sim = LBM("D3V19", (64, 30, 24), 0.8, E=(1e-4, 2e-5, 0.0), B=(0.0, 0.0, 1e-3), storage="f16")
    sim.set_geometry(torch.from_numpy(mask.reshape(-1)).cuda())
    sim.init_equilibrium()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        sim.step(7)
        ref_rho, ref_j = sim.moments()
        sim.moment_totals_static(out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] / ref_rho - 1) < 1e-12
        scale = max(np.abs(ref_j).max(), 1e-300)
        assert np.max(np.abs(got[1:] - ref_j)) <= 1e-12 * scale
    sim.close()
