"""Seeded synthetic inputs: flag fields, boundary set-ups and random states.

This module holds no lattice Boltzmann arithmetic.  It only draws geometry and
random numbers, and it serves both the CUDA path (tests, bench) and the
oracle (tests), so that both see identical inputs.

Workloads (sizes of the paper's lid-driven cavity, Sec. 5, and of the
channel / porous-media cases of the benchmark configurations):
  cavity(n)            n^3 lid-driven cavity, lid = +y face moving along x
  channel(dims)        periodic x and z, resting walls at -y/+y (Poiseuille)
  sphere_packing(...)  random non-overlapping spheres in a channel
  overlapping_spheres(...) random overlapping spheres (any porosity)
  batch_instances(...) many uneven channels with sphere packings and tau
  channel_samples(...) the learned warm start's samples: n^3 sphere-packed
                       channels with porosity and driving force per seed
"""
from __future__ import annotations

import os

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
    max_failures consecutive draws were rejected.  A cell is solid when its
    centre lies inside a sphere (distance <= r, periodic along x and z).
    """
    nx, ny, nz = dims
    flags = np.zeros((nz, ny, nx), np.uint8)
    target = (1.0 - porosity) * nx * ny * nz
    cen = np.zeros((0, 3))
    rad = np.zeros(0)
    fails = 0
    solid = 0
    while solid < target and fails < max_failures:
        r = int(rng.integers(rmin, rmax + 1))
        c = rng.uniform([0, 0, 0], [nx, ny, nz])
        if len(rad):
            d = np.abs(cen - c)
            d[:, 0] = np.minimum(d[:, 0], nx - d[:, 0])
            d[:, 2] = np.minimum(d[:, 2], nz - d[:, 2])
            if np.any(np.sqrt((d * d).sum(axis=1)) < r + rad):
                fails += 1
                continue
        fails = 0
        cen = np.vstack([cen, c])
        rad = np.append(rad, r)
        # stamp the sphere over its bounding box only (wrapped along x and z)
        xs = np.arange(int(np.floor(c[0] - r - 1)), int(np.ceil(c[0] + r + 1)) + 1)
        ys = np.arange(max(0, int(np.floor(c[1] - r - 1))), min(ny, int(np.ceil(c[1] + r + 1)) + 1))
        zs = np.arange(int(np.floor(c[2] - r - 1)), int(np.ceil(c[2] + r + 1)) + 1)
        xs = np.unique(xs % nx)
        zs = np.unique(zs % nz)
        dx = np.abs(xs + 0.5 - c[0])
        dx = np.minimum(dx, nx - dx)
        dz = np.abs(zs + 0.5 - c[2])
        dz = np.minimum(dz, nz - dz)
        dy = ys + 0.5 - c[1]
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) <= r * r
        sub = flags[np.ix_(zs, ys, xs)]
        solid += int(np.count_nonzero(inside & (sub == FLUID)))
        sub[inside] = NOSLIP
        flags[np.ix_(zs, ys, xs)] = sub
    return flags


def overlapping_spheres(rng: np.random.Generator, dims, porosity, rmin=2, rmax=6):
    """Solid spheres that may overlap (a Boolean model of a porous medium),
    periodic in x and z, added in batches until the fluid fraction is at most
    `porosity`; any fluid fraction down to zero is reachable, unlike the
    non-overlapping packing.  Integer radii uniform in [rmin, rmax]."""
    nx, ny, nz = dims
    solid = np.zeros((nz, ny, nx), bool)
    mean_vol = np.mean([4.0 / 3.0 * np.pi * r**3 for r in range(rmin, rmax + 1)])
    while (~solid).mean() > porosity:
        # enough spheres to close about half the remaining gap
        k = max(1, int(0.5 * ((~solid).mean() - porosity) * nx * ny * nz / mean_vol))
        for _ in range(k):
            r = int(rng.integers(rmin, rmax + 1))
            c = rng.uniform([0, 0, 0], [nx, ny, nz])
            xs = np.arange(int(np.floor(c[0] - r - 1)), int(np.ceil(c[0] + r + 1)) + 1) % nx
            zs = np.arange(int(np.floor(c[2] - r - 1)), int(np.ceil(c[2] + r + 1)) + 1) % nz
            ys = np.arange(max(0, int(np.floor(c[1] - r - 1))), min(ny, int(np.ceil(c[1] + r + 1)) + 1))
            xs, zs = np.unique(xs), np.unique(zs)
            dx = np.abs(xs + 0.5 - c[0])
            dx = np.minimum(dx, nx - dx)
            dz = np.abs(zs + 0.5 - c[2])
            dz = np.minimum(dz, nz - dz)
            dy = ys + 0.5 - c[1]
            inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) <= r * r
            sub = solid[np.ix_(zs, ys, xs)]
            solid[np.ix_(zs, ys, xs)] = sub | inside
    return np.where(solid, NOSLIP, FLUID).astype(np.uint8)


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


def channel_sample(seed: int, n: int = 64, f_lo: float = 5e-7, f_hi: float = 5e-6, por_lo: float = 0.7,
                   por_hi: float = 0.9):
    """One warm-start sample from default_rng(seed): porosity U[por_lo, por_hi],
    force U[f_lo, f_hi] along x, then the sphere packing of an n^3 channel."""
    rng = np.random.default_rng(seed)
    porosity = float(rng.uniform(por_lo, por_hi))
    force = float(rng.uniform(f_lo, f_hi))
    return sphere_packing(rng, (n, n, n), porosity), force


def channel_samples(seeds, n: int = 64, processes: int | None = None):
    """channel_sample for every seed, in order; a pool of spawned processes
    (no CUDA state is inherited) when there are many."""
    seeds = [int(s) for s in seeds]
    if processes == 1 or len(seeds) < 16:
        return [channel_sample(s, n) for s in seeds]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    procs = processes or min(len(seeds), os.cpu_count() or 1)
    # a worker that cannot start raises BrokenProcessPool here instead of hanging
    with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(channel_sample, seeds, [n] * len(seeds), chunksize=max(1, len(seeds) // (4 * procs))))
