"""Seeded synthetic inputs for the hybrid lattice Boltzmann scheme.

This module is the only code that the CUDA path and the CPU oracle both use:
it makes initial fields (density, order parameter, velocity) and holds none of
the scheme's arithmetic.  All randomness comes from splitmix64 of
(seed, site index), so every field is reproducible on any machine.

Workload recipes (the paper's test configurations, Sec. III, with the
parameter sets stated where they are used):
  * ``drop``          centred circular/spherical drop phi0 tanh((R - r)/xi);
  * ``spinodal``      i.i.d. uniform phi in [-amp, amp] (phase separation);
  * ``flat_interface`` two planar interfaces (periodic box) along x;
  * ``shear_wave``    u_x = U sin(2 pi y / Ly) over uniform phi.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """count doubles in [0, 1): splitmix64(seed * 2^32 + stream * 2^48 + site) >> 11."""
    base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) ^ (np.uint64(stream & 0xFFFF) << np.uint64(48))
    idx = np.arange(count, dtype=np.uint64) ^ base
    return (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def shape_of(dims: int, Lx: int, Ly: int, Lz: int = 1):
    return (Lz, Ly, Lx) if dims == 3 else (Ly, Lx)


def rest(dims: int, Lx: int, Ly: int, Lz: int = 1, n0: float = 1.0):
    """Uniform density n0 and zero velocity: (n[shape], u[dims, shape])."""
    shp = shape_of(dims, Lx, Ly, Lz)
    return np.full(shp, n0), np.zeros((dims,) + shp)


def spinodal(dims: int, Lx: int, Ly: int, Lz: int = 1, seed: int = 0, amp: float = 0.01):
    """phi i.i.d. uniform in [-amp, amp] from splitmix64(seed, site)."""
    shp = shape_of(dims, Lx, Ly, Lz)
    S = int(np.prod(shp))
    return (amp * (2.0 * uniform01(seed, S) - 1.0)).reshape(shp)


def drop(dims: int, Lx: int, Ly: int, Lz: int = 1, R: float = 16.0, phi0: float = 1.0,
         xi: float = 1.0, centre=None):
    """phi = phi0 tanh((R - r)/xi): positive inside a drop of radius R.

    The centre defaults to (Lx/2, Ly/2[, Lz/2]) in lattice coordinates; r is the
    plain Euclidean distance (the drop is assumed to fit in the box).
    """
    shp = shape_of(dims, Lx, Ly, Lz)
    if centre is None:
        centre = (Lx / 2.0, Ly / 2.0, Lz / 2.0)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shp], indexing="ij")
    coords = grids[::-1]  # x, y(, z)
    r2 = sum((coords[a] - centre[a]) ** 2 for a in range(dims))
    return phi0 * np.tanh((R - np.sqrt(r2)) / xi)


def flat_interface(dims: int, Lx: int, Ly: int, Lz: int = 1, phi0: float = 1.0,
                   xi: float = 1.0, x1=None, x2=None):
    """Two planar interfaces normal to x at x1 < x2 (default Lx/4, 3Lx/4):
    phi = phi0 [tanh((x - x1)/xi) - tanh((x - x2)/xi) - 1], +phi0 between them."""
    shp = shape_of(dims, Lx, Ly, Lz)
    x1 = Lx / 4.0 if x1 is None else x1
    x2 = 3.0 * Lx / 4.0 if x2 is None else x2
    x = np.arange(Lx, dtype=np.float64)
    prof = phi0 * (np.tanh((x - x1) / xi) - np.tanh((x - x2) / xi) - 1.0)
    return np.broadcast_to(prof, shp).copy()


def shear_wave(dims: int, Lx: int, Ly: int, Lz: int = 1, U: float = 1e-4):
    """Velocity u_x = U sin(2 pi y / Ly), other components zero: u[dims, shape]."""
    shp = shape_of(dims, Lx, Ly, Lz)
    u = np.zeros((dims,) + shp)
    y = np.arange(Ly, dtype=np.float64)
    prof = U * np.sin(2.0 * np.pi * y / Ly)
    if dims == 2:
        u[0] = prof[:, None]
    else:
        u[0] = prof[None, :, None]
    return u


def batch_instances(count: int = 512, seed: int = 0, side_min: int = 32, side_max: int = 256,
                    side_step: int = 16, force_fraction: float = 0.5):
    """Seeded descriptors of a batch of independent 2D drop instances.

    side uniform in {side_min, side_min + side_step, ..., side_max}, drop radius
    uniform in [6, side/3], and the first force_fraction of a seeded shuffle of
    the instances carry a body force.  Returns a list of dicts
    (side, R, forced).
    """
    nsides = (side_max - side_min) // side_step + 1
    u = uniform01(seed, 3 * count, stream=7).reshape(count, 3)
    sides = side_min + side_step * np.minimum((u[:, 0] * nsides).astype(int), nsides - 1)
    radii = 6.0 + u[:, 1] * (sides / 3.0 - 6.0)
    order = np.argsort(u[:, 2], kind="stable")
    forced = np.zeros(count, dtype=bool)
    forced[order[: int(round(force_fraction * count))]] = True
    return [dict(side=int(s), R=float(r), forced=bool(f)) for s, r, f in zip(sides, radii, forced)]
