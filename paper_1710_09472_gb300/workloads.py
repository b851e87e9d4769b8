"""Seeded synthetic inputs for the semiclassical LBM workloads.

This module holds no arithmetic of the method: it only builds geometries
(solid masks), initial fields and per-cell field samples from a counter-based
generator, so that the CUDA library, the oracle and the benchmark all read
the same inputs.  Arrays are C-ordered over ``shape`` = (ny, nx) in 2D and
(nz, ny, nx) in 3D, i.e. x is the fastest index.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  Obstacles follow a Boolean model: sphere
(disk) centres are i.i.d. uniform in the periodic box, and spheres are added
until the fluid fraction drops to the target porosity (the paper places
randomly "sorted" circles/spheres in Sec. 9.4 without naming a rule).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of SplitMix64 started at `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
    """Box-Muller normals from pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:count]
    return mean + std * z


def boolean_obstacles(shape, radius: float, porosity: float, seed: int, max_objects: int = 10_000_000):
    """Solid mask (uint8, 1 = solid) of overlapping disks (2D) or spheres (3D).

    Centres are uniform in the periodic box; a cell (at integer coordinates)
    is solid when its periodic distance to a centre is <= radius.  Objects are
    added one at a time until the fluid fraction is <= porosity.  Returns
    (mask, number_of_objects)."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    mask = np.zeros(shape, dtype=np.uint8)
    total = mask.size
    target_solid = int(np.ceil((1.0 - porosity) * total))
    solid = 0
    r = float(radius)
    ir = int(np.ceil(r))
    offs = np.arange(-ir, ir + 1)
    batch = 4096
    k = 0
    while solid < target_solid and k < max_objects:
        u = uniform01(seed, batch * nd, offset=k * nd).reshape(batch, nd)
        for b in range(batch):
            centre = u[b] * np.array(shape, dtype=np.float64)  # (z, y, x) order
            base = np.floor(centre).astype(np.int64)
            grids = []
            d2 = 0.0
            for ax in range(nd):
                coords = base[ax] + offs
                delta = coords - centre[ax]
                shp = [1] * nd
                shp[ax] = len(offs)
                d2 = d2 + (delta ** 2).reshape(shp)
                grids.append(np.mod(coords, shape[ax]))
            inside = d2 <= r * r + 1e-12
            idx = np.ix_(*grids)
            sub = mask[idx]
            newly = np.logical_and(inside, sub == 0)
            solid += int(newly.sum())
            sub[newly] = 1
            mask[idx] = sub
            k += 1
            if solid >= target_solid:
                break
    return mask, k


def channel_mask(shape):
    """Plane channel: solid rows y = 0 and y = ny-1, periodic elsewhere."""
    mask = np.zeros(shape, dtype=np.uint8)
    mask[..., 0, :] = 1
    mask[..., -1, :] = 1
    return mask


def end_walls_mask(shape):
    """Solid columns at x = 0 and x = nx-1 (a closed shock tube)."""
    mask = np.zeros(shape, dtype=np.uint8)
    mask[..., 0] = 1
    mask[..., -1] = 1
    return mask


def riemann_density(shape, rho_left: float, rho_right: float, x_split: int):
    rho = np.full(shape, rho_right, dtype=np.float64)
    rho[..., :x_split] = rho_left
    return rho


# --- the five workloads --------------------------------------------------------
# Each returns a dict with the geometry, the initial fields and the run
# parameters; the lattice is named by its paper label.

def poiseuille_32x64():
    shape = (64, 32)
    return dict(name="poiseuille-2d-32x64", vel="D2V9", shape=shape, solid=channel_mask(shape),
                rho=np.ones(shape), tau=0.8, E=(1e-6, 0.0, 0.0), B=(0.0, 0.0, 0.0), steps=5000)


def riemann_4096x8():
    shape = (8, 4096)
    return dict(name="riemann-2d-4096x8", vel="D2V9", shape=shape, solid=end_walls_mask(shape),
                rho=riemann_density(shape, 1.05, 1.0, 2048), tau=0.6, E=(0.0, 0.0, 0.0),
                B=(0.0, 0.0, 0.0), steps=2000)


def porous_3d(n: int = 256, radius: float = 6.0, porosity: float = 0.7, seed: int = 1,
              Ex: float = 1e-6, Bz: float = 0.0, tau: float = 0.8, steps: int = 20000):
    shape = (n, n, n)
    mask, count = boolean_obstacles(shape, radius, porosity, seed)
    return dict(name=f"porous-3d-{n}^3", vel="D3V19", shape=shape, solid=mask, n_objects=count,
                rho=np.ones(shape), tau=tau, E=(Ex, 0.0, 0.0), B=(0.0, 0.0, Bz), steps=steps)


def porous_2d_differentiable(n: int = 1024, radius: float = 8.0, porosity: float = 0.6, geom_seed: int = 2,
                             field_seed: int = 3, E_mean: float = 1e-6, E_std: float = 1e-7, tau: float = 0.7,
                             steps: int = 4000):
    shape = (n, n)
    mask, count = boolean_obstacles(shape, radius, porosity, geom_seed)
    Efield = np.zeros((2,) + shape, dtype=np.float32)
    Efield[0] = normal(field_seed, n * n, E_mean, E_std).reshape(shape).astype(np.float32)
    return dict(name=f"porous-2d-{n}^2-differentiable", vel="D2V9", shape=shape, solid=mask, n_objects=count,
                rho=np.ones(shape), tau=tau, Efield=Efield, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0),
                steps=steps, loss_window=500, checkpoint_every=100)


def porous_3d_512():
    shape = (512, 512, 512)
    mask, count = boolean_obstacles(shape, 10.0, 0.65, 5)
    return dict(name="porous-3d-512^3", vel="D3V19", shape=shape, solid=mask, n_objects=count,
                rho=np.ones(shape), tau=0.8, E=(2e-6, 0.0, 0.0), B=(0.0, 0.0, 5e-4), steps=10000)
