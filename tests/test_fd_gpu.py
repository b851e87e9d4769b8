"""GPU density <-> chemical-potential conversions (Sec. 9.1, Eq. rho-def-eq and
its inverse of Sec. 9.1.2) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("theta", [1.0 / 270.0, 0.1])
def test_density_and_mu_match_oracle(D, theta):
    """mu/theta spread over the classical series (< -30), the table (-30..60)
    and the Sommerfeld series (> 60): rho(mu) to 3e-7 relative (FP32 output)
    and mu(rho) of those densities to 1e-6 relative (or 1e-6 theta)."""
    from paper_1710_09472_gb300.lbm import density_from_mu, mu_from_density

    rng = np.random.default_rng(D * 10 + int(theta * 100))
    eta = np.concatenate([rng.uniform(-45, -30, 40), rng.uniform(-30, 60, 160), rng.uniform(60, 400, 60),
                          np.array([-30.0, 0.0, 60.0, 270.0])])
    mu = (eta * theta).astype(np.float32)
    rho_g = density_from_mu(D, theta, torch.from_numpy(mu).cuda()).cpu().numpy()
    rho_o = np.array([oracle.density_of_mu(D, theta, float(m)) for m in mu])
    rel = np.abs(rho_g / rho_o - 1)
    assert rel.max() < 3e-7, (rel.max(), eta[np.argmax(rel)])
    mu_g = mu_from_density(D, theta, torch.from_numpy(rho_g).cuda()).cpu().numpy()
    mu_o = np.array([oracle.mu_of_density(D, theta, float(r)) for r in rho_g])
    err = np.abs(mu_g - mu_o) / np.maximum(np.abs(mu_o), theta)
    assert err.max() < 1e-6, (err.max(), eta[np.argmax(err)])


def test_density_field_round_trip():
    """A density field of the 3D model (rho = 4.189 at mu = 1, Sec. 9.4) to
    mu and back, on a 64^3 field: mu within 1e-6 of 1 where rho is the
    equilibrium value, and rho recovered to 1e-6."""
    from paper_1710_09472_gb300.lbm import density_from_mu, mu_from_density

    theta = 1.0 / 270.0
    rho0 = oracle.density_of_mu(3, theta, 1.0)
    rho = torch.full((64 ** 3,), rho0, dtype=torch.float32, device="cuda")
    rho += 1e-3 * torch.rand(64 ** 3, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    rho[0] = rho0
    mu = mu_from_density(3, theta, rho)
    back = density_from_mu(3, theta, mu)
    assert abs(float(mu[0]) - 1.0) < 1e-6
    assert float(torch.max(torch.abs(back / rho - 1))) < 1e-6


def test_invalid_arguments():
    from paper_1710_09472_gb300._lib import LBMError
    from paper_1710_09472_gb300.lbm import density_from_mu, mu_from_density

    x = torch.ones(8, device="cuda")
    with pytest.raises(LBMError):
        density_from_mu(4, 0.1, x)
    with pytest.raises(LBMError):
        mu_from_density(2, -1.0, x)
    bad = torch.tensor([0.0, -1.0, float("inf"), 1.0], device="cuda")
    out = mu_from_density(2, 0.1, bad).cpu().numpy()
    assert np.all(np.isnan(out[:3])) and np.isfinite(out[3])
