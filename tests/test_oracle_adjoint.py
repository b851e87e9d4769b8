"""Pins of the oracle's adjoint (reverse sweep of the collide-and-stream step)
against central finite differences of the oracle's forward run, which the
physics tests pin independently.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl

THETA = 1.0 / 270.0


def _setup(vel, force):
    if vel == "D2V9":
        shape = (10, 12)
        mask, _ = wl.boolean_obstacles(shape, 2.0, 0.8, seed=21)
        B = (0.0, 0.0, 2e-2)
    else:
        shape = (5, 6, 7)
        mask, _ = wl.boolean_obstacles(shape, 1.5, 0.8, seed=22)
        B = (1e-2, -2e-2, 3e-2)
    D = len(shape)
    N = mask.size
    Efield = np.zeros((D,) + shape)
    Efield[0] = 1e-3 + 2e-4 * wl.normal(31, N).reshape(shape)
    Efield[1] = 3e-4 * wl.normal(32, N).reshape(shape)
    rho0 = 1.0 + 0.02 * wl.uniform01(33, N).reshape(shape)
    u0 = 0.01 * wl.normal(34, D * N).reshape((D,) + shape)
    wr = wl.normal(35, N).reshape(shape)
    wj = wl.normal(36, D * N).reshape((D,) + shape)
    return shape, mask, B, Efield, rho0, u0, wr, wj


def _loss(m, shape, mask, f0, Efield, T, t_begin, wr, wj):
    f = f0.copy()
    L = 0.0
    for t in range(1, T + 1):
        m.step(shape, mask, f, 1, Efield)
        if t > t_begin:
            rho, j, _ = m.moments(shape, mask, f)
            L += np.sum(wr * rho) + np.sum(wj * j)
    return L


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
@pytest.mark.parametrize("force", ["term", "shift"])
def test_adjoint_vs_finite_differences(vel, force):
    shape, mask, B, Efield, rho0, u0, wr, wj = _setup(vel, force)
    tau, T, t_begin = 0.75, 12, 6
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, B=B, force=force)
    f0 = m.init_equilibrium(shape, mask, rho0, u0)
    states = m.trajectory(shape, mask, f0, T, Efield)
    res = m.adjoint(shape, mask, states, t_begin, T, wr, wj, Efield)
    L0 = _loss(m, shape, mask, f0, Efield, T, t_begin, wr, wj)
    assert abs(res["loss"] - L0) < 1e-12 * max(1, abs(L0))

    fluid = np.argwhere(mask == 0)
    rng = np.random.default_rng(0)
    # per-cell E: a few fluid cells, every component
    for k in rng.choice(len(fluid), 4, replace=False):
        cell = tuple(fluid[k])
        for d in range(len(shape)):
            h = 1e-6
            Ep, Em = Efield.copy(), Efield.copy()
            Ep[(d,) + cell] += h
            Em[(d,) + cell] -= h
            fd = (_loss(m, shape, mask, f0, Ep, T, t_begin, wr, wj)
                  - _loss(m, shape, mask, f0, Em, T, t_begin, wr, wj)) / (2 * h)
            ad = res["gE"][(d,) + cell]
            assert abs(ad - fd) < 1e-6 * max(abs(fd), 1e-3), (cell, d, ad, fd)

    # B (every component that acts in this dimension) and tau
    comps = [2] if vel == "D2V9" else [0, 1, 2]
    for c in comps:
        h = 1e-6
        Bp, Bm = list(B), list(B)
        Bp[c] += h
        Bm[c] -= h
        mp = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, B=Bp, force=force)
        mm = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, B=Bm, force=force)
        fd = (_loss(mp, shape, mask, f0, Efield, T, t_begin, wr, wj)
              - _loss(mm, shape, mask, f0, Efield, T, t_begin, wr, wj)) / (2 * h)
        assert abs(res["gB"][c] - fd) < 1e-6 * max(abs(fd), 1e-3), (c, res["gB"][c], fd)
    h = 1e-6
    mp = oracle.Model(vel, "fd", THETA, 1.0, tau=tau + h, B=B, force=force)
    mm = oracle.Model(vel, "fd", THETA, 1.0, tau=tau - h, B=B, force=force)
    fd = (_loss(mp, shape, mask, f0, Efield, T, t_begin, wr, wj)
          - _loss(mm, shape, mask, f0, Efield, T, t_begin, wr, wj)) / (2 * h)
    assert abs(res["gtau"] - fd) < 1e-6 * max(abs(fd), 1e-3), (res["gtau"], fd)

    # initial populations along a random direction (a dot-product test of the
    # whole reverse sweep, streaming transpose included)
    v = rng.normal(size=f0.size)
    v.reshape(m.Q, -1)[:, mask.reshape(-1) == 1] = 0.0
    h = 1e-6
    fd = (_loss(m, shape, mask, f0 + h * v, Efield, T, t_begin, wr, wj)
          - _loss(m, shape, mask, f0 - h * v, Efield, T, t_begin, wr, wj)) / (2 * h)
    ad = float(res["lam0"] @ v)
    assert abs(ad - fd) < 1e-7 * max(abs(fd), 1.0), (ad, fd)
