"""Seeded synthetic inputs: flag fields, boundary set-ups and random states.

This module holds no lattice Boltzmann arithmetic.  It only draws geometry and
random numbers, and it serves both the CUDA path (tests, bench) and the
oracle (tests), so that both see identical inputs.

Workloads (sizes of the paper's lid-driven cavity, Sec. 5, and of the
channel / porous-media cases of the benchmark configurations):
  cavity(n)            n^3 lid-driven cavity, lid = +y face moving along x
  channel(dims)        periodic x and z, resting walls at -y/+y (Poiseuille)
  sphere_packing(...)  random non-overlapping spheres in a channel
  batch_instances(...) many uneven channels with sphere packings and tau
"""
from __future__ import annotations

import numpy as np

FLUID, NOSLIP, MOVING = 0, 1, 2


def cavity_bc():
    """Boundary set-up of the lid-driven cavity: walls everywhere, +y moves."""
    return dict(periodic=(0, 0, 0), face_bc=(NOSLIP, NOSLIP, NOSLIP, MOVING, NOSLIP, NOSLIP))


def channel_bc():
    """Channel: periodic along x and z, resting walls beyond -y and +y."""
    return dict(periodic=(1, 0, 1), face_bc=(NOSLIP,) * 6)


def random_flags(rng: np.random.Generator, dims, solid_fraction=0.2, moving_fraction=0.3):
    """Random per-cell flags (x fastest, shape (nz, ny, nx))."""
    nx, ny, nz = dims
    fl = (rng.random((nz, ny, nx)) < solid_fraction).astype(np.uint8)
    fl[(fl == NOSLIP) & (rng.random(fl.shape) < moving_fraction)] = MOVING
    return fl


def random_pdfs(rng: np.random.Generator, dims, amplitude=1e-2, flags=None):
    """Random shifted PDFs of shape (19, nz, ny, nx), zero in solid cells."""
    nx, ny, nz = dims
    f = rng.uniform(-amplitude, amplitude, (19, nz, ny, nx))
    if flags is not None:
        f *= (np.asarray(flags).reshape(nz, ny, nx) == FLUID)
    return f


def sphere_packing(rng: np.random.Generator, dims, porosity, rmin=2, rmax=6, max_failures=10_000):
    """Non-overlapping solid spheres in a channel (periodic in x and z).

    Integer radii uniform in [rmin, rmax]; centres uniform; a sphere is
    rejected when it overlaps another (periodic distance along x and z).
    Spheres are added until the solid fraction reaches 1 - porosity or
    max_failures consecutive draws were rejected.
    """
    nx, ny, nz = dims
    flags = np.zeros((nz, ny, nx), np.uint8)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    target = (1.0 - porosity) * nx * ny * nz
    spheres = []
    fails = 0
    solid = 0
    while solid < target and fails < max_failures:
        r = int(rng.integers(rmin, rmax + 1))
        c = rng.uniform([0, 0, 0], [nx, ny, nz])
        ok = True
        for (c2, r2) in spheres:
            d = np.abs(c - c2)
            d[0] = min(d[0], nx - d[0])
            d[2] = min(d[2], nz - d[2])
            if np.sqrt((d * d).sum()) < r + r2:
                ok = False
                break
        if not ok:
            fails += 1
            continue
        fails = 0
        spheres.append((c, r))
        dx = np.abs(x + 0.5 - c[0])
        dx = np.minimum(dx, nx - dx)
        dz = np.abs(z + 0.5 - c[2])
        dz = np.minimum(dz, nz - dz)
        dy = y + 0.5 - c[1]
        flags[dx * dx + dy * dy + dz * dz <= r * r] = NOSLIP
        solid = int((flags != FLUID).sum())
    return flags


def batch_instances(seed=1234, n=256, lo=16, hi=96, tau_lo=0.55, tau_hi=1.2,
                    por_lo=0.7, por_hi=0.9):
    """n independent channels: per-axis sizes uniform in [lo, hi], tau uniform in
    [tau_lo, tau_hi], a sphere packing of porosity uniform in [por_lo, por_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, 3))
        tau = float(rng.uniform(tau_lo, tau_hi))
        por = float(rng.uniform(por_lo, por_hi))
        out.append((dims, tau, sphere_packing(rng, dims, por)))
    return out
