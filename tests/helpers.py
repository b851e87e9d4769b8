"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs and measure the differences."""
from __future__ import annotations

import numpy as np

import oracle

THETA = 1.0 / 270.0

# Tolerances on rho and j after a run (relative L-inf: max|a-b| / max|b|).
# FP32 and FP16-deviation storage: the targets 1e-5 and 2e-3.  BF16 keeps 8
# mantissa bits, so one rounding of a stored deviation is already up to
# 2^-9 = 2e-3 of it; BF16 is held to 1.5e-2 and its measured error reported.
TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 1.5e-2}


def rel_linf(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b)))


def gpu_run(vel, shape, solid, tau, steps, storage="f32", force="term", E=(0, 0, 0), B=(0, 0, 0), rho=None,
            u=None, Efield=None):
    """Run the CUDA path; returns (rho[shape], j[D, *shape], totals, lbm)."""
    import torch

    from paper_1710_09472_gb300.lbm import LBM

    dims = tuple(reversed(shape))
    sim = LBM(vel, dims, tau, E=E, B=B, storage=storage, force=force)
    dev = torch.device("cuda")
    if solid is not None:
        sim.set_geometry(torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)).to(dev))
    if Efield is not None:
        sim.set_E_field(torch.from_numpy(np.ascontiguousarray(Efield, dtype=np.float32).reshape(-1)).to(dev))
    r = None if rho is None else torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32).reshape(-1)).to(dev)
    uu = None if u is None else torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32).reshape(-1)).to(dev)
    sim.init_equilibrium(r, uu)
    sim.step(steps)
    rho_d = torch.empty(sim.N, dtype=torch.float32, device=dev)
    j_d = torch.empty(sim.D * sim.N, dtype=torch.float32, device=dev)
    tot = sim.moments(rho_d, j_d)
    torch.cuda.synchronize()
    return (rho_d.cpu().numpy().reshape(shape), j_d.cpu().numpy().reshape((sim.D,) + tuple(shape)), tot, sim)


def oracle_run(vel, shape, solid, tau, steps, force="term", E=(0, 0, 0), B=(0, 0, 0), rho=None, u=None,
               Efield=None):
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, E=E, B=B, force=force)
    rho0 = np.ones(shape) if rho is None else np.asarray(rho, dtype=np.float64)
    f = m.init_equilibrium(shape, solid, rho0, None if u is None else np.asarray(u, dtype=np.float64))
    m.step(shape, solid, f, steps, None if Efield is None else np.asarray(Efield, dtype=np.float64))
    r, j, tot = m.moments(shape, solid, f)
    return r, j, tot, m, f
